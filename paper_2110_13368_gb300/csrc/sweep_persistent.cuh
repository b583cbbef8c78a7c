// Persistent line sweep for the step itself (included by sweeps.cu).
//
// Work: the lines of one axis that need a solve.  On a Dirichlet substrate
// a line whose other two coordinates touch the boundary lies entirely on the
// Dirichlet shell; its values are overwritten after every sweep and no later
// sweep reads them (the next sweep's lines through a shell voxel are either
// shell lines themselves or have that voxel as an end, whose input is
// replaced by the Dirichlet value).  Those lines are skipped and the shell is
// written once per step, after the z sweep, by k_shell_fill.  For the same
// reason the two end outputs of a Dirichlet line are not overwritten here.
//
// Each warp owns a column buffer of n_slots x 32 elements in shared memory
// (one column per lane, one lane per line) and walks a static list of
// 32-line blocks b0, b1, ...  The slot of element k alternates between k and
// n_slots-1-k from block to block (parity Q, a template parameter).  The back
// substitution of block b frees slots from the end of the line towards its
// start; under the alternation these are the slots of the *first* elements
// of block b+1, so:
//   - as soon as element k of block b has been back-substituted, element
//     n-1-k of block b+1 is copied (cp.async) into its slot;
//   - the forward elimination of block b+1 runs in the same loop, LAG
//     elements behind, on data that has had LAG iterations to arrive.
// The back substitution of b and the forward elimination of b+1 are two
// independent FMA chains, so every warp keeps two FP64 operations in flight
// while it needs no more shared memory than one block.  Only the first block
// of a warp is eliminated on its own, and only its last one back-substituted
// on its own.
//
// Shared-memory layout: element (slot, lane) sits in row `slot`; for the x
// sweep at column lane ^ ((slot mod G) * ROWS), so that both a lane's own
// column and the transposed copies hit every bank evenly, for the y and z
// sweeps at column lane.
//
// Global access: for the y and z sweeps adjacent lanes hold adjacent x, so
// each per-element access of a warp is one coalesced row.  For the x sweep
// the lanes hold 32 rows; copies and stores are transposed so that each
// instruction moves (32/G) rows x G consecutive elements = whole 32-byte
// sectors.
#pragma once

namespace bfvm {
namespace persistent {

// Group of G consecutive elements per loop iteration: 8 for both types (one
// 32-byte sector of FP32, two of FP64), so that per-group costs (waits,
// commits, pointer updates, boundary groups) are amortised over 8 elements.
template <typename T>
struct Groups {
    static constexpr int G = 8;
    static constexpr int ROWS = 32 / G;             // rows per transposed instruction
    static constexpr int LAG_GROUPS = sizeof(T) == 8 ? 3 : 4;
    // copy-ahead distance of a warp pair's F warp (sweep_pair.cuh); measured
    // on the 200^3 step: FP64 3 groups (289.5 us; 2: 310 us, 4: 292.5 us),
    // FP32 4 (8: 4 % slower)
    static constexpr int PAIR_LAG = sizeof(T) == 8 ? 3 : 4;
    // most warp pairs per CTA of the pair kernels (per-axis and one-launch):
    // FP64 is bound by the FP64 pipe with two pairs' warps per SMSP; the FP32
    // sweeps are latency-bound and take more warps.  Measured on the 200^3
    // FP32 step: 4 pairs 0.224 ms, 5 pairs 0.210 ms, 6 pairs 0.166 ms,
    // 8 pairs 0.192 ms.
    static constexpr int MAX_PAIRS = sizeof(T) == 8 ? 4 : 6;
    // most warp pairs per CTA of the per-axis pair kernel (k_sweep_pair);
    // FP32 at 8 pairs measured 12 % slower than at 6 (200^3 step)
    static constexpr int AXIS_PAIRS = MAX_PAIRS;
};

// Lines of one axis that need a solve, substrate by substrate: for a
// Dirichlet substrate the interior range of both other coordinates, else
// the full range.  first[s] is the index of substrate s's first line.
struct LineSet {
    int n_sub;
    const int64_t* first;   // [n_sub + 1]
    const int* lo_a;        // [n_sub] first value of the fast other coordinate
    const int* cnt_a;       // [n_sub] its count
    const int* lo_b;        // [n_sub] first value of the slow other coordinate
};

struct Line {
    int64_t base;      // first element (pitched layout)
    int s;             // substrate
    bool valid;        // a real line (the tail of the last block is padding)
    bool dir;          // Dirichlet substrate: both ends take the shell value
    double end0, end1; // input values of the two ends (Dirichlet)
    double inv_other;  // inverse of the other axes' scales (MODE 2)
};

template <typename T, int AXIS, int MODE>
__device__ __forceinline__ Line make_line(const SweepArgs<T>& A, const LineSet& S,
                                          const int64_t* first_s, int64_t line)
{
    Line L;
    const int64_t total = first_s[S.n_sub];
    L.valid = line < total;
    if (!L.valid) line = total - 1;
    int s = 0;
    while (s + 1 < S.n_sub && line >= first_s[s + 1]) ++s;
    L.s = s;
    int64_t t = line - first_s[s];
    const int ca = S.cnt_a[s];
    const int a = S.lo_a[s] + (int)(t % ca);
    const int b = S.lo_b[s] + (int)(t / ca);
    int ox = 0, oy = 0, oz = 0;
    if (AXIS == 0) {
        oy = a; oz = b;
        L.base = (((int64_t)s * A.nz + oz) * A.ny + oy) * A.pitch;
    } else if (AXIS == 1) {
        ox = a; oz = b;
        L.base = (((int64_t)s * A.nz + oz) * A.ny) * A.pitch + ox;
    } else {
        ox = a; oy = b;
        L.base = ((int64_t)s * A.nz * A.ny + oy) * A.pitch + ox;
    }
    L.dir = A.bc_kind[s] == BFVM_BC_DIRICHLET;
    double v0, v1;   // the ends' values: the boundary value, or a node's there
    end_values(A.ends, full_line<T, AXIS>(A, s, ox, oy, oz), A.bc_value[s], v0, v1);
    L.end0 = v0;
    L.end1 = v1;
    L.inv_other = 1.0;
    if (MODE >= 1) {
        const int64_t row = (int64_t)s * A.L;
        double sa, sb;
        if (AXIS == 0) {
            sa = A.sc_p[row + A.off_y + oy];
            sb = A.sc_p[row + A.off_z + oz];
        } else if (AXIS == 1) {
            sa = A.sc_p1[row + A.off_x + ox];
            sb = A.sc_p[row + A.off_z + oz];
        } else {
            sa = A.sc_p1[row + A.off_x + ox];
            sb = A.sc_p1[row + A.off_y + oy];
        }
        L.end0 = (v0 * sa * sb) * A.sc_p[row + A.axis_off];
        L.end1 = (v1 * sa * sb) * A.sc_p[row + A.axis_off + A.n - 1];
        if (MODE == 2 && AXIS == 2)
            L.inv_other = A.isc_p1[row + A.off_x + ox] * A.isc_p1[row + A.off_y + oy];
    }
    return L;
}

// Shared-memory coefficient rows of one substrate (this axis only).
template <typename T>
struct CoefRow {
    const T* a;      // forward: r (plain) or fa (rescaled)
    const T* a_lo;   // FP32 low parts of r
    const T* b;      // backward: cr (plain) or fb (rescaled)
    const T* b_lo;   // FP32 low parts of cr
    const double* o; // MODE 2: inverse output scale of this axis
    T c, c_lo;       // plain form: c
};

template <typename T, int AXIS, int MODE>
struct Sweeper {
    static constexpr int G = Groups<T>::G;
    static constexpr int ROWS = Groups<T>::ROWS;
    static constexpr int LG = Groups<T>::LAG_GROUPS;

    const SweepArgs<T>& A;
    T* W;                 // this warp's column buffer
    const T* fin;
    T* fout;
    int64_t stride;
    int n, ns, lane;

    // slot of element k under parity Q; since n_slots is a multiple of G the
    // slot's residue mod G is known from k mod G alone
    template <int Q>
    __device__ __forceinline__ int slot(int k) const { return Q ? (ns - 1 - k) : k; }
    template <int Q>
    __device__ __forceinline__ static constexpr int res(int kmod) { return Q ? (G - 1 - kmod) : kmod; }
    // element of lane/row l in slot s whose residue mod G is m; only the x
    // sweep (transposed copies) swizzles, the y and z sweeps keep lane l in
    // column l (every access path must agree on this)
    __device__ __forceinline__ T* at(int s, int l, int m) const
    {
        return W + s * 32 + (AXIS == 0 ? (l ^ (m * ROWS)) : l);
    }
    // this lane's element of the slot holding element k (k mod G == u)
    template <int Q>
    __device__ __forceinline__ T* own(int k, int u) const
    {
        return at(slot<Q>(k), lane, res<Q>(u));
    }

    __device__ __forceinline__ T fwd(const CoefRow<T>& C, T prev, T d, int k) const
    {
        if (MODE == 0) {
            if (sizeof(T) == 8) return fma(C.c, prev, d) * C.a[k];
            float t = comp_axpy((float)C.c, (float)C.c_lo, (float)prev, (float)d);
            return (T)__fmaf_rn(t, (float)C.a[k], __fmul_rn(t, (float)C.a_lo[k]));
        }
        return fma(C.a[k], prev, d);
    }

    __device__ __forceinline__ T bwd(const CoefRow<T>& C, T x, T w, int k) const
    {
        if (MODE == 0 && sizeof(T) == 4)
            return (T)comp_axpy((float)C.b[k], (float)C.b_lo[k], (float)x, (float)w);
        return fma(C.b[k], x, w);
    }

    __device__ __forceinline__ T out_value(const CoefRow<T>& C, const Line& L, T x, int k) const
    {
        if (MODE == 2) return (T)(((double)x * C.o[k]) * L.inv_other);
        return x;
    }

    // copy elements [gG, gG+G) of a block's lines into the slots of parity Q
    template <int Q>
    __device__ __forceinline__ void copy_group(const Line& ln, const int64_t* rb, int g) const
    {
        if (g * G >= n) return;
        if (AXIS == 0) {
            const int e = g * G + (lane % G);
            if (e < n) {
                const int s = slot<Q>(e);
                const int m = res<Q>(lane % G);
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int r = t * ROWS + lane / G;
                    cp_async_elem(at(s, r, m), fin + rb[r] + e);
                }
            }
        } else {
            const T* src = fin + ln.base + (int64_t)g * G * stride;
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (g * G + u < n) cp_async_elem(own<Q>(g * G + u, u), src + u * stride);
        }
    }

    // write out elements [hG, hG+G) of the current block (values in o[])
    template <int Q>
    __device__ __forceinline__ void store_group(const Line& L, const int64_t* rb, int h,
                                                const T* o) const
    {
        if (AXIS == 0) {
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (h * G + u < n) *own<Q>(h * G + u, u) = o[u];
            __syncwarp();
            const int k = h * G + (lane % G);
            if (k < n) {
                const int s = slot<Q>(k);
                const int m = res<Q>(lane % G);
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int r = t * ROWS + lane / G;
                    if (rb[r] >= 0) fout[rb[r] + k] = *at(s, r, m);
                }
            }
            __syncwarp();
        } else if (L.valid) {
            T* dst = fout + L.base + (int64_t)h * G * stride;
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (h * G + u < n) dst[u * stride] = o[u];
        }
    }

    // forward elimination of a whole block on its own (first block of a warp)
    template <int Q>
    __device__ __forceinline__ T forward_solo(const Line& L, const CoefRow<T>& C) const
    {
        T prev = (T)0;
        for (int g = 0; g * G < n; ++g) {
            T d[G];
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (g * G + u < n) d[u] = *own<Q>(g * G + u, u);
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int k = g * G + u;
                if (k < n) {
                    T dk = d[u];
                    if (L.dir && k == 0) dk = (T)L.end0;
                    if (L.dir && k == n - 1) dk = (T)L.end1;
                    prev = (k == 0 && MODE != 0) ? dk : fwd(C, prev, dk, k);
                    if (k < n - 1) *own<Q>(k, u) = prev;
                }
            }
        }
        return prev;
    }

    // back substitution of the last block of a warp on its own
    template <int Q>
    __device__ __forceinline__ void backward_solo(const Line& L, const CoefRow<T>& C, T x,
                                                  const int64_t* rb) const
    {
        const int h_top = (n - 1) / G;
        for (int h = h_top; h >= 0; --h) {
            T w[G], o[G];
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (h * G + u < n - 1) w[u] = *own<Q>(h * G + u, u);
#pragma unroll
            for (int u = G - 1; u >= 0; --u) {
                const int k = h * G + u;
                if (k < n) {
                    if (k < n - 1) x = bwd(C, x, w[u], k);
                    o[u] = out_value(C, L, x, k);
                }
            }
            store_group<Q>(L, rb, h, o);
        }
    }

    // Iteration groups jg in [j0, j1) of the interleaved loop in which both
    // groups are complete interior groups (no line end, no ragged tail) and
    // the copied group is complete: straight-line code with running
    // pointers, so every per-element offset is an immediate.
    template <int Q>
    __device__ __forceinline__ void fast_run(const Line& L, const CoefRow<T>& C, T& x,
                                             const Line& N, const CoefRow<T>& CN, T& prev,
                                             int j0, int j1, int h_top,
                                             const int64_t* rb_cur, const int64_t* rb_nxt) const
    {
        constexpr int P = 1 - Q;
        constexpr int SW = (AXIS == 0);          // swizzled columns (x sweep only)
        constexpr int RS = 32;                    // elements per slot row
        if (j0 >= j1) return;
        int lx[G];
#pragma unroll
        for (int m = 0; m < G; ++m) lx[m] = SW ? (lane ^ (m * ROWS)) : lane;
        // group h of block b occupies rows hb .. hb+G-1 (Q = 0, ascending k)
        // or ns-1-hb-(G-1) .. ns-1-hb (Q = 1, k descending in rows)
        int h = h_top - j0;
        int g = j0 - LG;
        T* rbw = W + (Q ? (ns - 1 - h * G) : h * G) * RS;   // row of k = hG
        T* rfd = W + (P ? (ns - 1 - g * G) : g * G) * RS;   // row of k = gG (block b+1)
        const T* cb = C.b + h * G;
        const T* ca = CN.a + g * G;
        const T* cbl = C.b_lo + h * G;
        const T* cal = CN.a_lo + g * G;
        const double* co = C.o + h * G;
        const int64_t sG = (int64_t)G * stride;
        T* pout = fout + L.base + (int64_t)h * G * stride;
        const T* psrc = fin + N.base + (int64_t)(ns / G - 1 - h) * sG;
        // x sweep: this lane's transposed rows and element offset
        int64_t rcur[G], rnxt[G];
        if (AXIS == 0) {
#pragma unroll
            for (int t = 0; t < G; ++t) {
                rcur[t] = rb_cur[t * ROWS + lane / G];
                rnxt[t] = rb_nxt[t * ROWS + lane / G];
            }
        }
        const int um = lane % G;
        // results of the previous group, stored one group late so that the
        // stores never wait for a DFMA that has only just been issued
        T po[G], pf[G];
        T* ppout = nullptr;
        T* prfd = nullptr;
        bool pending = false;
        for (int jg = j0; jg < j1; ++jg) {
            cp_async_wait<LG - 1>();
            __syncwarp();
            if (AXIS != 0 && pending) {
#pragma unroll
                for (int u = 0; u < G; ++u) prfd[(P ? -u : u) * RS + lx[res<P>(u)]] = pf[u];
                if (L.valid) {
                    T* p = ppout;
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        *p = po[u];
                        p += stride;
                    }
                }
            }
            T w[G], d[G], bb[G], aa[G], bl[G], al[G], o[G], f[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                w[u] = rbw[(Q ? -u : u) * RS + lx[res<Q>(u)]];
                d[u] = rfd[(P ? -u : u) * RS + lx[res<P>(u)]];
                bb[u] = cb[u];
                aa[u] = ca[u];
                if (MODE == 0 && sizeof(T) == 4) {
                    bl[u] = cbl[u];
                    al[u] = cal[u];
                }
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int ub = G - 1 - u;
                if (MODE == 0 && sizeof(T) == 4) {
                    x = (T)comp_axpy((float)bb[ub], (float)bl[ub], (float)x, (float)w[ub]);
                    float t = comp_axpy((float)CN.c, (float)CN.c_lo, (float)prev, (float)d[u]);
                    prev = (T)__fmaf_rn(t, (float)aa[u], __fmul_rn(t, (float)al[u]));
                } else if (MODE == 0) {
                    x = fma(bb[ub], x, w[ub]);
                    prev = fma(CN.c, prev, d[u]) * aa[u];
                } else {
                    x = fma(bb[ub], x, w[ub]);
                    prev = fma(aa[u], prev, d[u]);
                }
                o[ub] = (MODE == 2) ? (T)(((double)x * co[ub]) * L.inv_other) : x;
                f[u] = prev;
            }
            // element u of the copied group lands in row hG + (G-1-u) (Q = 0)
            // or ns-1-hG-(G-1-u) (Q = 1), i.e. rbw + (Q ? u-(G-1) : (G-1)-u) rows
            if (AXIS != 0) {
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    pf[u] = f[u];
                    po[u] = o[u];
                }
                prfd = rfd;
                ppout = pout;
                pending = true;
                const T* q = psrc;
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const int rowoff = Q ? (u - (G - 1)) : ((G - 1) - u);
                    cp_async_elem(rbw + rowoff * RS + lx[res<P>(u)], q);
                    q += stride;
                }
            } else {
#pragma unroll
                for (int u = 0; u < G; ++u) rfd[(P ? -u : u) * RS + lx[res<P>(u)]] = f[u];
#pragma unroll
                for (int u = 0; u < G; ++u) rbw[(Q ? -u : u) * RS + lx[res<Q>(u)]] = o[u];
                __syncwarp();
                // transposed store: element k = hG + um of rows t*ROWS + lane/G
                const int ks = h * G + um;
                const T* srow = rbw + (Q ? -um : um) * RS;
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int r = t * ROWS + lane / G;
                    const T v = srow[r ^ ((Q ? (G - 1 - um) : um) * ROWS)];
                    if (rcur[t] >= 0) fout[rcur[t] + ks] = v;
                }
                __syncwarp();
                // transposed copy of e-group eg = ns/G-1-h into the same rows
                const int e = (ns / G - 1 - h) * G + um;
                const int rowoff = Q ? (um - (G - 1)) : ((G - 1) - um);
                T* drow = rbw + rowoff * RS;
                const int mres = Q ? um : (G - 1 - um);   // residue of that row
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int r = t * ROWS + lane / G;
                    cp_async_elem(drow + (r ^ (mres * ROWS)), fin + rnxt[t] + e);
                }
            }
            cp_async_commit();
            // advance: h decreases, g increases
            --h;
            ++g;
            rbw += (Q ? G : -G) * RS;
            rfd += (P ? -G : G) * RS;
            cb -= G;
            ca += G;
            cbl -= G;
            cal += G;
            co -= G;
            pout -= sG;
            psrc += sG;
        }
        if (AXIS != 0 && pending) {
#pragma unroll
            for (int u = 0; u < G; ++u) prfd[(P ? -u : u) * RS + lx[res<P>(u)]] = pf[u];
            if (L.valid) {
                T* p = ppout;
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    *p = po[u];
                    p += stride;
                }
            }
        }
    }

    // Back substitution of block b (parity Q, value x = its last
    // intermediate) interleaved with the forward elimination of block b+1
    // (parity !Q), LAG = LG*G elements behind.  Returns b+1's last
    // intermediate.
    template <int Q>
    __device__ __forceinline__ T interleaved(const Line& L, const CoefRow<T>& C, T x,
                                             const Line& N, const CoefRow<T>& CN,
                                             const int64_t* rb_cur, const int64_t* rb_nxt) const
    {
        constexpr int P = 1 - Q;
        const int gcount = (n + G - 1) / G;
        const int h_top = gcount - 1;
        T prev = (T)0;
        // interior range of iteration groups for the straight-line loop:
        // h = h_top - jg in [0, h_top) with (h+1)G <= n-1, g = jg - LG in
        // [1, gcount-1) with (g+1)G <= n-1, copied e-group complete
        int j_fast0 = LG + 1;
        int j_fast1 = gcount + LG;
        {
            const int hmax = (n - 1) / G - 1;           // (h+1)G <= n-1
            const int gmax = (n - 1) / G - 1;           // (g+1)G <= n-1
            const int hmin = ns / G - n / G;            // (ns/G - h) G <= n
            // jg >= h_top - hmax, jg <= h_top - hmin, jg <= gmax + LG
            j_fast0 = max(j_fast0, h_top - min(hmax, h_top - 1));
            j_fast1 = min(j_fast1, min(h_top - max(hmin, 0), gmax + LG) + 1);
            if (j_fast0 >= j_fast1) j_fast0 = j_fast1 = -1;
        }
        // iteration group jg: back substitution of group h = h_top - jg of
        // block b, forward elimination of group g = jg - LG of block b+1.
        // The group of block b+1 that lands in the slots freed by group h is
        // e-group ns/G - 1 - h.
        for (int jg = 0; jg < gcount + LG; ++jg) {
            const int h = h_top - jg;
            const int g = jg - LG;
            // copies of e-groups <= g are complete once at most LG - 1 of the
            // newest commit groups are still pending
            if (g >= 0) {
                cp_async_wait<LG - 1>();
                __syncwarp();
            }
            if (jg == j_fast0) {
                fast_run<Q>(L, C, x, N, CN, prev, j_fast0, j_fast1, h_top, rb_cur, rb_nxt);
                jg = j_fast1 - 1;
                continue;
            }
            T w[G], d[G], o[G];
            if (h >= 0) {
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (h * G + u < n - 1) w[u] = *own<Q>(h * G + u, u);
            }
            if (g >= 0 && g < gcount) {
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (g * G + u < n) d[u] = *own<P>(g * G + u, u);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                // one step of each chain
                if (h >= 0) {
                    const int k = h * G + (G - 1 - u);
                    if (k < n) {
                        if (k < n - 1) x = bwd(C, x, w[G - 1 - u], k);
                        o[G - 1 - u] = out_value(C, L, x, k);
                    }
                }
                if (g >= 0 && g < gcount) {
                    const int k = g * G + u;
                    if (k < n) {
                        T dk = d[u];
                        if (N.dir && k == 0) dk = (T)N.end0;
                        if (N.dir && k == n - 1) dk = (T)N.end1;
                        prev = (k == 0 && MODE != 0) ? dk : fwd(CN, prev, dk, k);
                        if (k < n - 1) *own<P>(k, u) = prev;
                    }
                }
            }
            if (h >= 0) {
                store_group<Q>(L, rb_cur, h, o);
                copy_group<P>(N, rb_nxt, ns / G - 1 - h);
            }
            cp_async_commit();
        }
        return prev;
    }
};

// Dynamic shared memory: [coefficients of all substrates for this axis]
// [MODE 2 output scales] [line-set prefix] [per warp: column buffer,
// 2 x 32 row bases].
template <typename T, int AXIS, int MODE>
__global__ void __launch_bounds__(256, 1) k_sweep_persistent(SweepArgs<T> A, LineSet S,
                                                             int64_t n_blocks, int n_slots)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const int n = A.n;
    const int ns = n_slots;
    const int n_sub = A.n_sub;

    const int ncoef = (MODE == 0 ? (sizeof(T) == 4 ? 4 : 2) : 2);
    T* cbase = reinterpret_cast<T*>(smem_raw);
    const int per_sub = ncoef * n;
    const size_t coef_bytes = (size_t)n_sub * per_sub * sizeof(T);
    double* obase = reinterpret_cast<double*>(smem_raw + ((coef_bytes + 15) & ~(size_t)15));
    const size_t o_bytes = (MODE == 2) ? (size_t)n_sub * n * sizeof(double) : 0;
    int64_t* first_s = reinterpret_cast<int64_t*>(
        reinterpret_cast<unsigned char*>(obase) + ((o_bytes + 15) & ~(size_t)15));
    unsigned char* warp_area = reinterpret_cast<unsigned char*>(first_s) +
                               (((size_t)(n_sub + 1) * 8 + 15) & ~(size_t)15);
    for (int i = threadIdx.x; i < n_sub * n; i += blockDim.x) {
        const int s = i / n, k = i % n;
        const int64_t src = (int64_t)s * A.L + A.axis_off + k;
        T* dst = cbase + (size_t)s * per_sub;
        if (MODE == 0) {
            dst[k] = A.r[src];
            dst[n + k] = A.cr[src];
            if (sizeof(T) == 4) {
                dst[2 * n + k] = A.r_lo[src];
                dst[3 * n + k] = A.cr_lo[src];
            }
        } else {
            dst[k] = (T)A.fa[src];
            dst[n + k] = (T)A.fb[src];
            if (MODE == 2) obase[(size_t)s * n + k] = A.isc_p1[src];
        }
    }
    for (int i = threadIdx.x; i <= n_sub; i += blockDim.x) first_s[i] = S.first[i];
    __syncthreads();

    const size_t warp_bytes = (size_t)ns * 32 * sizeof(T) + 2 * 32 * sizeof(int64_t);
    unsigned char* my = warp_area + (size_t)warp * warp_bytes;
    T* W = reinterpret_cast<T*>(my);
    int64_t* rowbase = reinterpret_cast<int64_t*>(my + (size_t)ns * 32 * sizeof(T));

    const int64_t tw = (int64_t)gridDim.x * warps;
    int64_t b = (int64_t)blockIdx.x * warps + warp;
    if (b >= n_blocks) return;

    Sweeper<T, AXIS, MODE> sw{A, W, A.in, A.field,
                              AXIS == 0 ? 1 : (AXIS == 1 ? A.pitch : (int64_t)A.ny * A.pitch),
                              n, ns, lane};
    auto coef_row = [&](int s) {
        CoefRow<T> C;
        const T* r = cbase + (size_t)s * per_sub;
        C.a = r;
        C.b = r + n;
        C.a_lo = r + 2 * n;
        C.b_lo = r + 3 * n;
        C.o = obase + (size_t)s * n;
        C.c = (MODE == 0) ? A.cvec[s * 3 + AXIS] : (T)0;
        C.c_lo = (MODE == 0 && sizeof(T) == 4) ? A.cvec_lo[s * 3 + AXIS] : (T)0;
        return C;
    };
    // rowbase[0..31]: stores of the current block (-1 = padding row);
    // rowbase[32..63]: copies of the block being loaded (padding rows read a
    // valid row, their results are dropped)
    int64_t* rb_cur = rowbase;
    int64_t* rb_nxt = rowbase + 32;

    Line cur = make_line<T, AXIS, MODE>(A, S, first_s, b * 32 + lane);
    rb_nxt[lane] = cur.base;
    rb_cur[lane] = cur.valid ? cur.base : -1;
    __syncwarp();
    for (int g = 0; g * sw.G < n; ++g) sw.template copy_group<0>(cur, rb_nxt, g);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    CoefRow<T> C = coef_row(cur.s);
    T x = sw.template forward_solo<0>(cur, C);
    int par = 0;
    for (;;) {
        const int64_t nb = b + tw;
        if (nb >= n_blocks) {
            if (par == 0) sw.template backward_solo<0>(cur, C, x, rb_cur);
            else sw.template backward_solo<1>(cur, C, x, rb_cur);
            break;
        }
        Line nxt = make_line<T, AXIS, MODE>(A, S, first_s, nb * 32 + lane);
        CoefRow<T> CN = coef_row(nxt.s);
        __syncwarp();
        rb_nxt[lane] = nxt.base;
        __syncwarp();
        if (par == 0) x = sw.template interleaved<0>(cur, C, x, nxt, CN, rb_cur, rb_nxt);
        else x = sw.template interleaved<1>(cur, C, x, nxt, CN, rb_cur, rb_nxt);
        cp_async_wait<0>();
        __syncwarp();
        rb_cur[lane] = nxt.valid ? nxt.base : -1;
        __syncwarp();
        b = nb;
        cur = nxt;
        C = CN;
        par ^= 1;
    }
}

// Dirichlet shell after the z sweep: every voxel of the outer layer of a
// Dirichlet substrate gets the value times the field's current scale (state
// p + 1 of all three axes), or the plain value when the step renormalised.
template <typename T>
__global__ void k_shell_fill(T* __restrict__ field, int nx, int ny, int nz, int n_sub,
                             int64_t pitch, const int32_t* __restrict__ kind,
                             const double* __restrict__ value, int64_t L,
                             const double* __restrict__ sc, int zfaces)
{
    // faces enumerated as: z planes (2 nx ny), y rows of the other planes
    // (2 nx nz), x columns (2 ny nz); overlaps are written twice with the
    // same value.  A z plane is written only where zfaces marks it as a
    // boundary (bit 0: z = 0, bit 1: z = nz - 1): neither in the 2-D variant,
    // only the grid's own end planes on a z-slab of a decomposed grid.
    const int64_t fz = 2 * (int64_t)nx * ny, fy = 2 * (int64_t)nx * nz, fx = 2 * (int64_t)ny * nz;
    const int64_t per = fz + fy + fx;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= per * n_sub) return;
    const int s = (int)(e / per);
    if (kind[s] != BFVM_BC_DIRICHLET) return;
    int64_t t = e % per;
    int x, y, z;
    if (t < fz) {
        const bool hi = (t / ((int64_t)nx * ny)) != 0;
        if (!(zfaces & (hi ? 2 : 1))) return;
        x = (int)(t % nx); y = (int)((t / nx) % ny); z = hi ? nz - 1 : 0;
    } else if ((t -= fz) < fy) {
        x = (int)(t % nx); z = (int)((t / nx) % nz); y = (t / ((int64_t)nx * nz)) ? ny - 1 : 0;
    } else {
        t -= fy;
        y = (int)(t % ny); z = (int)((t / ny) % nz); x = (t / ((int64_t)ny * nz)) ? nx - 1 : 0;
    }
    double v = value[s];
    if (sc) {
        const double* q = sc + (int64_t)s * L;
        v = v * (q[x] * q[nx + y] * q[nx + ny + z]);
    }
    field[(((int64_t)s * nz + z) * ny + y) * pitch + x] = (T)v;
}

}  // namespace persistent
}  // namespace bfvm
