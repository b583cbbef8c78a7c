// Persistent, software-pipelined line sweep (included by sweeps.cu).
//
// Each warp owns a column buffer of n_slots x 32 elements in shared memory
// (one column per lane, one lane per line) and walks a static list of
// 32-line blocks.  Per block:
//   1. wait for the block's elements (copied in by cp.async while the
//      previous block was being back-substituted);
//   2. forward elimination in place, eight elements at a time with the next
//      eight already loaded into registers (the chain is one dependent FMA
//      per element in the rescaled FP64 form);
//   3. back substitution four elements (one group) at a time; each finished
//      group is written out, and its shared-memory slots are immediately
//      refilled with the next block's elements.
// The slot of element k alternates between k and n_slots-1-k from one block
// to the next.  The back substitution frees slots from the end of the line
// towards its start, and with the alternation those are exactly the slots
// of the *first* elements of the next block, so the data needed first
// arrives first and the forward pass of the next block rarely waits.
//
// Global access patterns: for the y and z sweeps adjacent lanes hold
// adjacent x, so each per-element access of a warp is one coalesced row.
// For the x sweep the 32 lanes hold 32 consecutive rows; copies and stores
// are transposed so that each instruction moves (32/G) rows x G consecutive
// elements = whole 32-byte sectors (G = 32 bytes / element size).
#pragma once

namespace bfvm {
namespace persistent {

template <typename T>
struct Groups {
    static constexpr int G = 32 / (int)sizeof(T);   // elements per 32-byte sector
    static constexpr int ROWS = 32 / G;             // rows per transposed instruction
};

struct LaneLine {
    int64_t base;      // first element of the line (pitched layout)
    int s;             // substrate
    bool valid;        // a real line (the tail of the last block is padding)
    bool dir;          // Dirichlet substrate
    bool shell;        // the whole line lies on the Dirichlet shell
    double v;          // Dirichlet value (0 in the adjoint)
    double kline;      // Dirichlet value times the other axes' scales
    double inv_other;  // inverse of the other axes' scales (MODE 2)
};

template <typename T, int AXIS, int MODE, int DIR>
__device__ __forceinline__ LaneLine lane_line(const SweepArgs<T>& A, int64_t line)
{
    LaneLine L;
    L.valid = line < A.n_lines;
    if (!L.valid) line = A.n_lines - 1;
    int ox = 0, oy = 0, oz = 0;
    int64_t t = line;
    if (AXIS == 0) {
        oy = (int)(t % A.ny); t /= A.ny;
        oz = (int)(t % A.nz); L.s = (int)(t / A.nz);
        L.base = line * A.pitch;
        L.shell = (oy == 0 || oy == A.ny - 1 || oz == 0 || oz == A.nz - 1);
    } else if (AXIS == 1) {
        ox = (int)(t % A.nx); t /= A.nx;
        oz = (int)(t % A.nz); L.s = (int)(t / A.nz);
        L.base = (((int64_t)L.s * A.nz + oz) * A.ny) * A.pitch + ox;
        L.shell = (ox == 0 || ox == A.nx - 1 || oz == 0 || oz == A.nz - 1);
    } else {
        ox = (int)(t % A.nx); t /= A.nx;
        oy = (int)(t % A.ny); L.s = (int)(t / A.ny);
        L.base = ((int64_t)L.s * A.nz * A.ny + oy) * A.pitch + ox;
        L.shell = (ox == 0 || ox == A.nx - 1 || oy == 0 || oy == A.ny - 1);
    }
    L.dir = A.bc_kind[L.s] == BFVM_BC_DIRICHLET;
    double v = (DIR == 2) ? 0.0 : A.bc_value[L.s];
    L.v = v;
    L.kline = v;
    L.inv_other = 1.0;
    if (MODE >= 1) {
        const int64_t row = (int64_t)L.s * A.L;
        if (AXIS == 0)
            L.kline = v * A.sc_p[row + A.off_y + oy] * A.sc_p[row + A.off_z + oz];
        else if (AXIS == 1)
            L.kline = v * A.sc_p1[row + A.off_x + ox] * A.sc_p[row + A.off_z + oz];
        else {
            L.kline = v * A.sc_p1[row + A.off_x + ox] * A.sc_p1[row + A.off_y + oy];
            if (MODE == 2)
                L.inv_other = A.isc_p1[row + A.off_x + ox] * A.isc_p1[row + A.off_y + oy];
        }
    }
    return L;
}

// fl(a*u + v) for an FP32 coefficient held as a = hi + lo, with one final
// rounding of an almost exact value: the product error comes from an FMA
// (TwoProduct) and the sum error from Knuth's TwoSum; explicit _rn
// intrinsics keep the compiler from contracting them.
__device__ __forceinline__ float comp_axpy(float a_hi, float a_lo, float u, float v)
{
    float p = __fmul_rn(a_hi, u);
    float pe = __fmaf_rn(a_hi, u, -p);
    float s = __fadd_rn(p, v);
    float z = __fsub_rn(s, p);
    float se = __fadd_rn(__fsub_rn(p, __fsub_rn(s, z)), __fsub_rn(v, z));
    float corr = __fmaf_rn(a_lo, u, __fadd_rn(pe, se));
    return __fadd_rn(s, corr);
}

template <typename T>
__device__ __forceinline__ void cp8(T* dst, const T* src);
template <>
__device__ __forceinline__ void cp8<double>(double* dst, const double* src)
{
    cp_async_elem(dst, src);
}
template <>
__device__ __forceinline__ void cp8<float>(float* dst, const float* src)
{
    cp_async_elem(dst, src);
}

template <typename T, int AXIS, int MODE, int DIR>
__global__ void __launch_bounds__(256, 1) k_sweep_persistent(SweepArgs<T> A, int64_t n_blocks,
                                                             int n_slots)
{
    constexpr int G = Groups<T>::G;
    constexpr int ROWS = Groups<T>::ROWS;
    constexpr int FC = 8;   // forward chunk (elements)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const int n = A.n;
    const int ns = n_slots;
    T* __restrict__ W = reinterpret_cast<T*>(smem_raw) + (size_t)warp * ns * 32;
    const int64_t tw = (int64_t)gridDim.x * warps;
    int64_t b = (int64_t)blockIdx.x * warps + warp;
    if (b >= n_blocks) return;

    const T* __restrict__ fin = A.in;
    T* __restrict__ fout = A.field;
    const int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? A.pitch : (int64_t)A.ny * A.pitch);

    auto slot = [&](int q, int k) { return q ? (ns - 1 - k) : k; };

    // copy elements [4g, 4g + G) of the lines of block bb into slots of parity q
    auto prefetch_group = [&](int64_t bb, const LaneLine& ln, int q, int g) {
        if (AXIS == 0) {
            const int rsub = lane / G;
            const int e = g * G + (lane % G);
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const int row = t * ROWS + rsub;
                int64_t line = bb * 32 + row;
                if (line >= A.n_lines) line = A.n_lines - 1;
                if (e < n) cp8<T>(W + (size_t)slot(q, e) * 32 + row, fin + line * A.pitch + e);
            }
        } else {
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int e = g * G + u;
                if (e < n) cp8<T>(W + (size_t)slot(q, e) * 32 + lane, fin + ln.base + e * stride);
            }
        }
    };

    int q = 0;
    LaneLine cur = lane_line<T, AXIS, MODE, DIR>(A, b * 32 + lane);
    for (int g = 0; g < ns / G; ++g) prefetch_group(b, cur, 0, g);
    cp_async_commit();

    const int64_t srow = 0;  // coefficient rows are per lane (substrate)
    (void)srow;
    for (;;) {
        const int64_t nb = b + tw;
        const bool has_next = nb < n_blocks;
        LaneLine nxt = has_next ? lane_line<T, AXIS, MODE, DIR>(A, nb * 32 + lane) : cur;
        cp_async_wait<0>();
        __syncwarp();

        const int64_t row = (int64_t)cur.s * A.L + A.axis_off;
        // ------------------------------------------------ forward
        T prev = (T)0;
        {
            T d0[FC], a0[FC], a0l[FC];
            auto load_chunk = [&](int k0, T* d, T* a, T* al) {
#pragma unroll
                for (int u = 0; u < FC; ++u) {
                    const int k = k0 + u;
                    if (k < n) {
                        d[u] = W[(size_t)slot(q, k) * 32 + lane];
                        if (MODE == 0) {
                            a[u] = A.r[row + k];
                            if (sizeof(T) == 4) al[u] = A.r_lo[row + k];
                        } else {
                            a[u] = (T)A.fa[row + k];
                        }
                    }
                }
            };
            load_chunk(0, d0, a0, a0l);
            const T c = MODE == 0 ? A.cvec[cur.s * 3 + AXIS] : (T)0;
            const T c_lo = (MODE == 0 && sizeof(T) == 4) ? A.cvec_lo[cur.s * 3 + AXIS] : (T)0;
            for (int k0 = 0; k0 < n; k0 += FC) {
                T d1[FC], a1[FC], a1l[FC];
                load_chunk(k0 + FC, d1, a1, a1l);
#pragma unroll
                for (int u = 0; u < FC; ++u) {
                    const int k = k0 + u;
                    if (k < n) {
                        T d = d0[u];
                        const bool end = (k == 0 || k == n - 1);
                        if (cur.dir && (end || (DIR == 1 && cur.shell))) {
                            if (MODE == 0) d = (T)cur.kline;
                            else d = (T)(cur.kline * A.sc_p[row + k]);
                        }
                        if (MODE == 0) {
                            if (sizeof(T) == 8) {
                                prev = fma(c, prev, d) * a0[u];
                            } else {
                                float t = comp_axpy((float)c, (float)c_lo, (float)prev, (float)d);
                                prev = (T)__fmaf_rn(t, (float)a0[u], __fmul_rn(t, (float)a0l[u]));
                            }
                        } else {
                            prev = fma(a0[u], prev, d);
                        }
                        W[(size_t)slot(q, k) * 32 + lane] = prev;
                    }
                }
#pragma unroll
                for (int u = 0; u < FC; ++u) {
                    d0[u] = d1[u];
                    a0[u] = a1[u];
                    a0l[u] = a1l[u];
                }
            }
        }

        // ------------------------------------------------ backward
        {
            const int h_top = (n - 1) / G;
            T wv0[G], b0[G], b0l[G];
            double so0[G];
            auto load_group = [&](int h, T* wv, T* bb, T* bl, double* so) {
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const int k = h * G + u;
                    if (h >= 0 && k < n) {
                        wv[u] = W[(size_t)slot(q, k) * 32 + lane];
                        if (MODE == 0) {
                            bb[u] = A.cr[row + k];
                            if (sizeof(T) == 4) bl[u] = A.cr_lo[row + k];
                        } else {
                            bb[u] = (T)A.fb[row + k];
                        }
                        if (MODE == 1) so[u] = A.sc_p1[row + k];
                        if (MODE == 2) so[u] = A.isc_p1[row + k];
                    }
                }
            };
            load_group(h_top, wv0, b0, b0l, so0);
            T x = prev;
            for (int h = h_top; h >= 0; --h) {
                T wv1[G], b1[G], b1l[G];
                double so1[G];
                load_group(h - 1, wv1, b1, b1l, so1);
                T o[G];
#pragma unroll
                for (int u = G - 1; u >= 0; --u) {
                    const int k = h * G + u;
                    if (k < n) {
                        if (k < n - 1) {
                            if (MODE == 0 && sizeof(T) == 4)
                                x = (T)comp_axpy((float)b0[u], (float)b0l[u], (float)x, (float)wv0[u]);
                            else
                                x = fma(b0[u], x, wv0[u]);
                        }
                        // output value of element k
                        const bool end = (k == 0 || k == n - 1);
                        bool ov = false;
                        if (DIR == 0) ov = cur.dir && (cur.shell || end);
                        if (DIR == 2) ov = cur.dir && cur.shell;
                        T out;
                        if (ov) {
                            if (DIR == 2) out = (T)0;
                            else if (MODE == 1) out = (T)(cur.kline * so0[u]);
                            else out = (T)cur.v;   // plain, or renormalised back to plain
                        } else if (MODE == 2) {
                            out = (T)(((double)x * so0[u]) * cur.inv_other);
                        } else {
                            out = x;
                        }
                        o[u] = out;
                    }
                }
                // write the group out
                if (AXIS == 0) {
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        const int k = h * G + u;
                        if (k < n) W[(size_t)slot(q, k) * 32 + lane] = o[u];
                    }
                    __syncwarp();
                    const int rsub = lane / G;
                    const int k = h * G + (lane % G);
#pragma unroll
                    for (int t = 0; t < G; ++t) {
                        const int r = t * ROWS + rsub;
                        const int64_t line = b * 32 + r;
                        if (k < n && line < A.n_lines)
                            fout[line * A.pitch + k] = W[(size_t)slot(q, k) * 32 + r];
                    }
                    __syncwarp();
                } else {
#pragma unroll
                    for (int u = 0; u < G; ++u) {
                        const int k = h * G + u;
                        if (k < n && cur.valid) fout[cur.base + k * stride] = o[u];
                    }
                }
                // refill the freed slots with the next block's elements
                if (has_next) prefetch_group(nb, nxt, q ^ 1, ns / G - 1 - h);
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    wv0[u] = wv1[u];
                    b0[u] = b1[u];
                    b0l[u] = b1l[u];
                    so0[u] = so1[u];
                }
            }
        }
        cp_async_commit();
        if (!has_next) break;
        b = nb;
        cur = nxt;
        q ^= 1;
    }
}

}  // namespace persistent
}  // namespace bfvm
