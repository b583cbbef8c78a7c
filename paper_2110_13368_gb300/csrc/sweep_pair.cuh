// Warp-pair line sweep for FP64 (included by sweeps.cu after
// sweep_persistent.cuh, whose LineSet / Line / make_line it reuses).
//
// The FP64 pipe of an SMSP only reaches its issue rate with two warps
// feeding it, but one 32-line block of 200 doubles per lane fills 51 KB of
// shared memory, so only four such blocks fit per SM.  Here each column
// buffer is shared by a pair of warps:
//   - warp F of the pair copies the elements of a block into the buffer and
//     runs its forward elimination;
//   - warp B of the pair runs the back substitution of the previous block
//     on the same buffer and writes the results out.
// The slot of element k alternates between k and n_slots-1-k from block to
// block, so the slots that B frees (from the end of the line backwards)
// are exactly those of the first elements of F's next block.  Both warps
// walk the same iteration count per block; after each group of G elements
// they meet at a named barrier (one per pair): B has finished reading and
// writing its group, so F may refill those slots.  F's forward runs LAG
// groups behind its copies.  A block's last intermediate passes from F to B
// through shared memory at another barrier.
//
// Every barrier is reached the same number of times by both warps of a
// pair: the block list, group count and lag are the same for both, and no
// warp leaves the loop early.
#pragma once

namespace bfvm {
namespace persistent {

// 16-byte vector of the element type
template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
    using type = double2;
};
template <>
struct Vec16<float> {
    using type = float4;
};

// BBAR: B meets F at the pair barrier between reading a group and solving
// it (true), or after solving it (false; see b_block)
// DUAL: B also writes every output to A.field2 (the adjoint's replay keeps
// the raw z solve and starts the next step from a copy of it)
template <typename T, int AXIS, int MODE, int LAG = Groups<T>::PAIR_LAG, bool BBAR = true,
          bool DUAL = false>
struct PairSweeper {
    static constexpr int G = Groups<T>::G;
    static constexpr int ROWS = Groups<T>::ROWS;
    static constexpr int LG = LAG;   // copy-ahead distance of F, in groups

    const SweepArgs<T>& A;
    T* W;
    const T* fin;
    T* fout;
    int64_t stride;
    int n, ns, lane;
    int bar_id;

    __device__ __forceinline__ void pair_bar() const
    {
        asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
    }
    template <int Q>
    __device__ __forceinline__ int slot(int k) const { return Q ? (ns - 1 - k) : k; }
    template <int Q>
    __device__ __forceinline__ static constexpr int res(int kmod) { return Q ? (G - 1 - kmod) : kmod; }
    __device__ __forceinline__ T* at(int s, int l) const { return W + s * 32 + l; }

    // x lines (AXIS 0) are contiguous in memory, so each lane copies,
    // eliminates and writes its own line.  The G elements of group g of a
    // lane lie together in the 32 G slots that elements [gG, gG+G) occupy in
    // the y/z layout (so the slot schedule is the same for every axis), as
    // 16-byte chunks whose order within the lane is swizzled so that the
    // 16-byte accesses of a quarter-warp fall on distinct banks.  Copies are
    // 16-byte cp.async, shared reads and writes 16-byte vectors, and B
    // writes its outputs with 32-byte (FP64) or 16-byte (FP32) stores.  Rows
    // start on 32-byte boundaries (the pitch is a multiple of 4 elements),
    // and a chunk that starts inside a line ends inside its row.
    static constexpr int CW = 16 / (int)sizeof(T);   // elements per chunk
    static constexpr int NCH = G / CW;               // chunks per lane and group
    using V16 = typename Vec16<T>::type;
    __device__ __forceinline__ int xswz() const { return (lane / (8 / NCH)) % NCH; }
    template <int Q>
    __device__ __forceinline__ T* xgrp(int g) const
    {
        return W + (Q ? (ns / G - 1 - g) : g) * (G * 32) + lane * G;
    }
    template <int Q>
    __device__ __forceinline__ T* xel(int k) const
    {
        const int u = k % G;
        return xgrp<Q>(k / G) + CW * ((u / CW) ^ xswz()) + u % CW;
    }
    template <int Q>
    __device__ __forceinline__ T* own(int k, int u) const
    {
        if (AXIS == 0) return xel<Q>(k);
        return at(slot<Q>(k), lane);
    }
    // chunks c of group g (x lines): 16-byte reads and writes
    __device__ __forceinline__ void x_read(const T* grp, T (&v)[G]) const
    {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const V16 q = *reinterpret_cast<const V16*>(grp + CW * (c ^ xswz()));
            const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int i = 0; i < CW; ++i) v[c * CW + i] = e[i];
        }
    }
    __device__ __forceinline__ void x_write_chunk(T* grp, int c, const T* v) const
    {
        V16 q;
        T* e = reinterpret_cast<T*>(&q);
#pragma unroll
        for (int i = 0; i < CW; ++i) e[i] = v[i];
        *reinterpret_cast<V16*>(grp + CW * (c ^ xswz())) = q;
    }
    // B's outputs of a whole group of an x line: two 32-byte (FP64) or two
    // 16-byte (FP32) stores
    __device__ __forceinline__ void x_store_group(T* dst, const T (&o)[G]) const
    {
        if (sizeof(T) == 8) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * h),
                             "d"((double)o[4 * h]), "d"((double)o[4 * h + 1]),
                             "d"((double)o[4 * h + 2]), "d"((double)o[4 * h + 3])
                             : "memory");
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                *reinterpret_cast<float4*>(dst + 4 * h) =
                    make_float4((float)o[4 * h], (float)o[4 * h + 1], (float)o[4 * h + 2],
                                (float)o[4 * h + 3]);
        }
    }

    // F: copy elements [gG, gG+G) of a block into the slots of parity Q
    template <int Q>
    __device__ __forceinline__ void copy_group(const Line& ln, const int64_t* rb, int g) const
    {
        if (g * G >= n) return;
        if (AXIS == 0) {
            if (!ln.valid) return;
            const T* src = fin + ln.base + g * G;
            T* d = xgrp<Q>(g);
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                if (g * G + c * CW < n) cp_async_16(d + CW * (c ^ xswz()), src + c * CW);
        } else {
            const T* src = fin + ln.base + (int64_t)g * G * stride;
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (g * G + u < n) cp_async_elem(own<Q>(g * G + u, u), src + u * stride);
        }
    }

    // One forward / backward recurrence step.  Plain form (MODE 0):
    // d'_k = (d_k + c d'_{k-1}) r_k, x_k = d'_k + (c r_k) x_{k+1}; in FP32
    // every coefficient is an unevaluated hi + lo pair and each step is a
    // hi + lo multiply-add (comp_axpy).  Rescaled form: one FMA each.
    __device__ __forceinline__ T fwd_op(const CoefRow<T>& C, T prev, T d, int k) const
    {
        return fwd_val(C, prev, d, C.a[k], (MODE == 0 && sizeof(T) == 4) ? C.a_lo[k] : (T)0);
    }
    // the same step with the element's coefficients already in registers.
    // EXACT (FP32, c exactly representable: c_lo = 0): fl(c prev + d), the
    // single rounding of one FMA
    template <bool EXACT = false>
    __device__ __forceinline__ T fwd_val(const CoefRow<T>& C, T prev, T d, T a, T a_lo) const
    {
        if (MODE != 0) return fma(a, prev, d);
        if (sizeof(T) == 8) return fma(C.c, prev, d) * a;
        const float t = EXACT ? __fmaf_rn((float)C.c, (float)prev, (float)d)
                              : comp_axpy((float)C.c, (float)C.c_lo, (float)prev, (float)d);
        return (T)__fmaf_rn(t, (float)a, __fmul_rn(t, (float)a_lo));
    }
    __device__ __forceinline__ T bwd_op(const CoefRow<T>& C, T x, T w, int k) const
    {
        return bwd_val(x, w, C.b[k], (MODE == 0 && sizeof(T) == 4) ? C.b_lo[k] : (T)0);
    }
    __device__ __forceinline__ T bwd_val(T x, T w, T b, T b_lo) const
    {
        if (MODE == 0 && sizeof(T) == 4)
            return (T)comp_axpy((float)b, (float)b_lo, (float)x, (float)w);
        return fma(b, x, w);
    }

    // B's inputs of one interior group, read ahead into registers: the
    // group's intermediates (written by F in the previous phase) and its
    // backward coefficients
    struct BIn {
        T w[G], b[G], bl[G];
    };
    template <int Q>
    __device__ __forceinline__ void bwd_load(const CoefRow<T>& C, int h, BIn& in) const
    {
        constexpr bool LO = MODE == 0 && sizeof(T) == 4;
        const int k0 = h * G;
        if (AXIS == 0) x_read(xgrp<Q>(h), in.w);
        const T* p = W + slot<Q>(k0) * 32;
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (AXIS != 0) in.w[u] = p[off<Q>(u)];
            in.b[u] = C.b[k0 + u];
            in.bl[u] = LO ? C.b_lo[k0 + u] : (T)0;
        }
    }

    // F: forward elimination of group g (parity Q); prev carries the chain
    template <int Q>
    __device__ __forceinline__ void fwd_group(const Line& L, const CoefRow<T>& C, T& prev,
                                              int g) const
    {
        // FP64: coefficients read with the elements, ahead of the chain
        constexpr bool HOIST = sizeof(T) == 8;
        T d[G], ca[G];
#pragma unroll
        for (int u = 0; u < G; ++u)
            if (g * G + u < n) {
                d[u] = *own<Q>(g * G + u, u);
                if (HOIST) ca[u] = C.a[g * G + u];
            }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int k = g * G + u;
            if (k < n) {
                T dk = d[u];
                if (L.dir && k == 0) dk = (T)L.end0;
                if (L.dir && k == n - 1) dk = (T)L.end1;
                const T nk = HOIST ? fwd_val(C, prev, dk, ca[u], (T)0) : fwd_op(C, prev, dk, k);
                if (MODE == 0) prev = nk;
                else prev = (k == 0) ? dk : nk;
                if (k < n - 1) *own<Q>(k, u) = prev;
            }
        }
    }

    // Column of element k0+u relative to row slot<Q>(k0) (compile-time u)
    template <int Q>
    __device__ __forceinline__ int off(int u) const
    {
        return (Q ? -u : u) * 32 + lane;
    }

    // Interior groups: all G elements exist, none is the line's last and
    // (forward) none its first, so no element needs a test and every
    // offset is a constant from one row pointer.
    template <int Q>
    __device__ __forceinline__ void copy_fast(const Line& ln, const int64_t (&rv)[G], int g) const
    {
        if (AXIS == 0) {
            if (!ln.valid) return;
            const T* src = fin + ln.base + g * G;
            T* d = xgrp<Q>(g);
#pragma unroll
            for (int c = 0; c < NCH; ++c) cp_async_16(d + CW * (c ^ xswz()), src + c * CW);
        } else {
            T* p = W + slot<Q>(g * G) * 32;
            const T* src = fin + ln.base + (int64_t)g * G * stride;
#pragma unroll
            for (int u = 0; u < G; ++u) cp_async_elem(p + off<Q>(u), src + u * stride);
        }
    }

    // The group's coefficients are read into registers with its elements,
    // before the chain: read inside it, each read would wait for the store
    // of the previous element (the two may alias, as far as the compiler
    // knows), and the shared-memory latency would sit on the chain.
    template <int Q>
    __device__ __forceinline__ void fwd_fast(const CoefRow<T>& C, T& prev, int g) const
    {
        constexpr bool LO = MODE == 0 && sizeof(T) == 4;
        T* p = AXIS == 0 ? xgrp<Q>(g) : W + slot<Q>(g * G) * 32;
        T d[G], ca[G], cl[G];
        if (AXIS == 0) x_read(p, d);
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (AXIS != 0) d[u] = p[off<Q>(u)];
            ca[u] = C.a[g * G + u];
            cl[u] = LO ? C.a_lo[g * G + u] : (T)0;
        }
        if (LO && C.c_lo == (T)0) fwd_chain<Q, true>(C, prev, p, d, ca, cl);
        else fwd_chain<Q, false>(C, prev, p, d, ca, cl);
    }
    template <int Q, bool EXACT>
    __device__ __forceinline__ void fwd_chain(const CoefRow<T>& C, T& prev, T* p, T (&d)[G],
                                              const T (&ca)[G], const T (&cl)[G]) const
    {
#pragma unroll
        for (int u = 0; u < G; ++u) {
            prev = fwd_val<EXACT>(C, prev, d[u], ca[u], cl[u]);
            if (AXIS == 0) {
                d[u] = prev;
                if (u % CW == CW - 1) x_write_chunk(p, u / CW, d + (u - (CW - 1)));
            } else {
                p[off<Q>(u)] = prev;
            }
        }
    }

    template <int Q>
    __device__ __forceinline__ void bwd_fast(const Line& L, const CoefRow<T>& C, T& x, int h,
                                             const int64_t (&rv)[G], const BIn& in) const
    {
        const int k0 = h * G;
        T o[G];
#pragma unroll
        for (int u = G - 1; u >= 0; --u) {
            x = bwd_val(x, in.w[u], in.b[u], in.bl[u]);
            o[u] = (MODE == 2) ? (T)(((double)x * C.o[k0 + u]) * L.inv_other) : x;
        }
        if (AXIS == 0) {
            if (L.valid) {
                x_store_group(fout + L.base + k0, o);
                if (DUAL) x_store_group(A.field2 + L.base + k0, o);
            }
        } else if (L.valid) {
            T* dst = fout + L.base + (int64_t)k0 * stride;
#pragma unroll
            for (int u = 0; u < G; ++u) dst[u * stride] = o[u];
            if (DUAL) {
                T* dst2 = A.field2 + L.base + (int64_t)k0 * stride;
#pragma unroll
                for (int u = 0; u < G; ++u) dst2[u * stride] = o[u];
            }
        }
    }

    // Row bases of transposed accesses: none in this layout (kept so that
    // the callers' row tables stay the same for every axis)
    __device__ __forceinline__ void load_rows(const int64_t* rb, int64_t (&rv)[G]) const
    {
#pragma unroll
        for (int t = 0; t < G; ++t) rv[t] = 0;   // no transposed accesses (any axis)
    }

    // F: forward elimination of a whole block on its own (the pair's first)
    template <int Q>
    __device__ __forceinline__ T f_solo(const Line& L, const CoefRow<T>& C) const
    {
        const int gcount = (n + G - 1) / G;
        const int f_hi = (n - 1) / G;
        T prev = (T)0;
        for (int g = 0; g < gcount; ++g) {
            if (g >= 1 && g < f_hi) fwd_fast<Q>(C, prev, g);
            else fwd_group<Q>(L, C, prev, g);
        }
        return prev;
    }

    // F: copies and forward elimination of block L (parity Q) while B
    // back-substitutes the previous block; one pair barrier per group.
    // `iters` (default gcount + LG) is the number of barrier meetings: the
    // step kernel pairs blocks of different line lengths and passes the
    // larger count to both warps; iterations past this block's groups only
    // meet the barrier.
    template <int Q>
    __device__ __forceinline__ T f_block(const Line& L, const CoefRow<T>& C, const int64_t* rb,
                                         const int64_t (&rv)[G], int iters = -1) const
    {
        const int gcount = (n + G - 1) / G;
        const int h_top = gcount - 1;
        const int f_hi = (n - 1) / G;   // forward groups [1, f_hi) are interior
        const int c_hi = n / G;         // copy groups [0, c_hi) are full
        if (iters < 0) iters = gcount + LG;
        T prev = (T)0;
        for (int jg = 0; jg < iters; ++jg) {
            const int g = jg - LG;
            if (g >= 0) {
                cp_async_wait<LG - 1>();
                __syncwarp();
                if (g >= 1 && g < f_hi) fwd_fast<Q>(C, prev, g);
                else fwd_group<Q>(L, C, prev, g);
            }
            pair_bar();                                  // B is done with group h_top - jg
            if (jg <= h_top) {
                if (jg < c_hi) copy_fast<Q>(L, rv, jg);
                else copy_group<Q>(L, rb, jg);
            }
            cp_async_commit();
        }
        return prev;
    }

    struct NoRelease {
        __device__ void operator()() const {}
    };

    // B: back substitution of block L (parity Q); with `paired`, the group
    // loop meets F at the pair barrier `iters` times (default gcount + LG).
    // `rel` runs once after the last group's stores have been issued: in the
    // first iteration that has no group left (F is still eliminating its
    // last groups then), else after the loop.
    //
    // With BBAR, B reads a group's inputs into registers before it meets F
    // at the pair barrier and runs the group's chain after it: the group's
    // slots are free once read (B's outputs go to global memory), and F
    // arrives at the barrier at the end of its own chain, so B's chain fills
    // the FP64 pipe while F issues its copies and reads its next group
    // (200^3 FP64 step 301 -> 292 us).  The batched step, whose tasks pair
    // lines of unequal length, measured faster with the chain before the
    // barrier (5.1e10 against 4.8e10 updates/s), and takes BBAR = false.
    template <int Q, typename Rel = NoRelease>
    __device__ __forceinline__ void b_block(const Line& L, const CoefRow<T>& C, T& x,
                                            const int64_t* rb, const int64_t (&rv)[G],
                                            bool paired, int iters = -1,
                                            const Rel& rel = Rel()) const
    {
        const int gcount = (n + G - 1) / G;
        const int h_top = gcount - 1;
        const int b_hi = (n - 1) / G;   // backward groups [0, b_hi) are interior
        if (!paired) iters = gcount;
        else if (iters < 0) iters = gcount + LG;
        bool released = false;
        BIn in;
        for (int jg = 0; jg < iters; ++jg) {
            const int h = h_top - jg;
            if (h >= 0) {
                if (h < b_hi) bwd_load<Q>(C, h, in);
                else bwd_load_edge<Q>(C, h, in);
                if (!BBAR) bwd_solve<Q>(L, C, x, h, b_hi, rv, in);
            } else if (!released) {
                rel();
                released = true;
            }
            if (paired) pair_bar();                      // group h released to F
            if (BBAR && h >= 0) bwd_solve<Q>(L, C, x, h, b_hi, rv, in);
        }
        if (!released) rel();
    }

    template <int Q>
    __device__ __forceinline__ void bwd_solve(const Line& L, const CoefRow<T>& C, T& x, int h,
                                              int b_hi, const int64_t (&rv)[G],
                                              const BIn& in) const
    {
        if (h < b_hi) bwd_fast<Q>(L, C, x, h, rv, in);
        else bwd_group<Q>(L, C, x, h, in);
    }

    // B: inputs of the line's last group (elements below n - 1 only)
    template <int Q>
    __device__ __forceinline__ void bwd_load_edge(const CoefRow<T>& C, int h, BIn& in) const
    {
        constexpr bool LO = MODE == 0 && sizeof(T) == 4;
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int k = h * G + u;
            if (k < n - 1) {
                in.w[u] = *own<Q>(k, u);
                in.b[u] = C.b[k];
                in.bl[u] = LO ? C.b_lo[k] : (T)0;
            }
        }
    }

    // B: back substitution of the line's last group (parity Q) and its output
    template <int Q>
    __device__ __forceinline__ void bwd_group(const Line& L, const CoefRow<T>& C, T& x, int h,
                                              const BIn& in) const
    {
        T o[G];
#pragma unroll
        for (int u = G - 1; u >= 0; --u) {
            const int k = h * G + u;
            if (k < n) {
                if (k < n - 1) x = bwd_val(x, in.w[u], in.b[u], in.bl[u]);
                o[u] = (MODE == 2) ? (T)(((double)x * C.o[k]) * L.inv_other) : x;
            }
        }
        if (AXIS == 0) {
            if (L.valid) {
                T* dst = fout + L.base + h * G;
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (h * G + u < n) dst[u] = o[u];
                if (DUAL) {
                    T* dst2 = A.field2 + L.base + h * G;
#pragma unroll
                    for (int u = 0; u < G; ++u)
                        if (h * G + u < n) dst2[u] = o[u];
                }
            }
        } else if (L.valid) {
            T* dst = fout + L.base + (int64_t)h * G * stride;
#pragma unroll
            for (int u = 0; u < G; ++u)
                if (h * G + u < n) dst[u * stride] = o[u];
            if (DUAL) {
                T* dst2 = A.field2 + L.base + (int64_t)h * G * stride;
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (h * G + u < n) dst2[u * stride] = o[u];
            }
        }
    }
};

// Dynamic shared memory: [coefficients of all substrates, this axis]
// [MODE 2 output scales] [line-set prefix] [per pair: column buffer,
// 2 x 32 row bases of each warp (4 x 32), 32 chain hand-over values].
template <typename T, int AXIS, int MODE, bool DUAL = false>
__global__ void __launch_bounds__(64 * Groups<T>::AXIS_PAIRS, 1) k_sweep_pair(SweepArgs<T> A, LineSet S,
                                                       int64_t n_blocks, int n_slots)
{
    constexpr int G = Groups<T>::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int pairs = blockDim.x >> 6;
    // warps p and p + pairs form pair p: with four pairs the F warps sit on
    // the four SMSPs (warp % 4), so the pipe is fed from all of them also
    // while the partner warps wait (a pair's first and last block)
    const int pair = warp % pairs;
    const bool is_b = warp >= pairs;     // B: back substitution; F: copies + forward
    const int n = A.n;
    const int ns = n_slots;
    const int n_sub = A.n_sub;

    const int ncoef = (MODE == 0 && sizeof(T) == 4) ? 4 : 2;   // FP32: hi and lo parts
    T* cbase = reinterpret_cast<T*>(smem_raw);
    const int per_sub = ncoef * n;
    const size_t coef_bytes = (size_t)n_sub * per_sub * sizeof(T);
    double* obase = reinterpret_cast<double*>(smem_raw + ((coef_bytes + 15) & ~(size_t)15));
    const size_t o_bytes = (MODE == 2) ? (size_t)n_sub * n * sizeof(double) : 0;
    int64_t* first_s = reinterpret_cast<int64_t*>(
        reinterpret_cast<unsigned char*>(obase) + ((o_bytes + 15) & ~(size_t)15));
    unsigned char* pair_area = reinterpret_cast<unsigned char*>(first_s) +
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

    const size_t pair_bytes = (size_t)ns * 32 * sizeof(T) + 4 * 32 * sizeof(int64_t) +
                              32 * sizeof(T);
    unsigned char* my = pair_area + (size_t)pair * pair_bytes;
    T* W = reinterpret_cast<T*>(my);
    int64_t* rbF = reinterpret_cast<int64_t*>(my + (size_t)ns * 32 * sizeof(T));  // [32] copy rows
    int64_t* rbB = rbF + 64;                                                       // [32] store rows
    T* handover = reinterpret_cast<T*>(rbF + 128);

    const int64_t tp = (int64_t)gridDim.x * pairs;
    const int64_t b0 = (int64_t)blockIdx.x * pairs + pair;
    if (b0 >= n_blocks) return;   // both warps of the pair leave together
    const int64_t nb = (n_blocks - 1 - b0) / tp + 1;   // blocks of this pair

    PairSweeper<T, AXIS, MODE, Groups<T>::PAIR_LAG, true, DUAL> sw{A, W, A.in, A.field,
                                  AXIS == 0 ? 1 : (AXIS == 1 ? A.pitch : (int64_t)A.ny * A.pitch),
                                  n, ns, lane, 1 + pair};
    auto coef_row = [&](int s) {
        CoefRow<T> C;
        const T* r = cbase + (size_t)s * per_sub;
        C.a = r;
        C.b = r + n;
        C.a_lo = (ncoef == 4) ? r + 2 * n : r;
        C.b_lo = (ncoef == 4) ? r + 3 * n : r;
        C.o = obase + (size_t)s * n;
        C.c = (MODE == 0) ? A.cvec[s * 3 + AXIS] : (T)0;
        C.c_lo = (ncoef == 4) ? A.cvec_lo[s * 3 + AXIS] : (T)0;
        return C;
    };
    const int gcount = (n + G - 1) / G;

    if (!is_b) {
        // ------------------------------------------------------- warp F
        Line cur = make_line<T, AXIS, MODE>(A, S, first_s, b0 * 32 + lane);
        rbF[lane] = cur.base;
        __syncwarp();
        for (int g = 0; g < gcount; ++g) sw.template copy_group<0>(cur, rbF, g);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        T prev = sw.template f_solo<0>(cur, coef_row(cur.s));
        handover[lane] = prev;
        sw.pair_bar();                                  // hand-over of block 0
        int64_t rv[G];
        for (int64_t k = 1; k < nb; ++k) {
            Line nxt = make_line<T, AXIS, MODE>(A, S, first_s, (b0 + k * tp) * 32 + lane);
            CoefRow<T> CN = coef_row(nxt.s);
            __syncwarp();
            rbF[lane] = nxt.base;
            __syncwarp();
            sw.load_rows(rbF, rv);
            if (k & 1) prev = sw.template f_block<1>(nxt, CN, rbF, rv);
            else prev = sw.template f_block<0>(nxt, CN, rbF, rv);
            cp_async_wait<0>();
            handover[lane] = prev;
            sw.pair_bar();                              // hand-over of block k
        }
    } else {
        // ------------------------------------------------------- warp B
        sw.pair_bar();                                  // hand-over of block 0
        Line cur = make_line<T, AXIS, MODE>(A, S, first_s, b0 * 32 + lane);
        CoefRow<T> C = coef_row(cur.s);
        T x = handover[lane];
        rbB[lane] = cur.valid ? cur.base : -1;
        __syncwarp();
        int64_t rv[G];
        sw.load_rows(rbB, rv);
        for (int64_t k = 1; k < nb; ++k) {
            // parity of the block B finishes: that of block k-1
            if ((k - 1) & 1) sw.template b_block<1>(cur, C, x, rbB, rv, true);
            else sw.template b_block<0>(cur, C, x, rbB, rv, true);
            sw.pair_bar();                              // hand-over of block k
            x = handover[lane];
            cur = make_line<T, AXIS, MODE>(A, S, first_s, (b0 + k * tp) * 32 + lane);
            C = coef_row(cur.s);
            __syncwarp();
            rbB[lane] = cur.valid ? cur.base : -1;
            __syncwarp();
            sw.load_rows(rbB, rv);
        }
        if ((nb - 1) & 1) sw.template b_block<1>(cur, C, x, rbB, rv, false);
        else sw.template b_block<0>(cur, C, x, rbB, rv, false);
    }
}

}  // namespace persistent
}  // namespace bfvm
