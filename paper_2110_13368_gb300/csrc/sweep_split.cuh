// Split (partitioned) line solve of one axis in the plain Thomas form, for
// axes whose lines are too few to fill the GPU with one thread (or one
// 32-line block) per line: the 2-D variant, and lines too long for the
// shared-memory kernels.  Included by sweeps.cu after its SweepArgs.
//
// Both recurrences of the solve (Sec. 2, Eq. 1 discretised per axis) are
// first-order and affine:
//   forward   d'_k = r_k d_k + m_k d'_{k-1},     m_k = c r_k  (the table cr)
//   backward  x_k  = d'_k + m_k x_{k+1}.
// A line of n elements is cut into segments [k0, k1) of `seg` elements.  Run
// from a zero incoming value, a segment's forward gives f_k, and the true
// d'_k = f_k + G_k D, where D is the true d' just before the segment and
// G_k = prod_{j=k0..k} m_j; likewise the backward from zero gives g_k and the
// true x_k = g_k + S_k X, X the true x just after the segment and
// S_k = prod_{j=k..k1-1} m_j.  G and S depend on the coefficients only and
// are tabulated at create (CoefTables::sg / sl).  The D of every segment
// follows from the segments' last f values by the same affine rule, and the
// X from the first g values, so a step runs three launches per axis, one
// thread per (segment, line):
//   1. forward from zero; f in place; the segment's last f to the exchange;
//   2. D by a scan over the earlier segments; the backward from zero on the
//      corrected d'; g in place; the segment's first g to the exchange;
//   3. X by a scan over the later segments; x = g + S X, Dirichlet ends set.
// This is the textbook algebra of the recurrence, not an approximation: it
// differs from the sequential solve by rounding only.  Threads of a warp
// take consecutive lines of one segment, so y and z accesses are coalesced
// rows.  An x line is contiguous, so a warp's 32 segments of 32 rows are
// staged through shared memory (a 32 x seg tile, copied row by row with
// consecutive lanes on consecutive elements) and each lane then walks its
// own row in the tile; the line count is padded to a multiple of 32 so that
// a warp never straddles two segments.
// In FP32 every table is an unevaluated hi + lo pair and every update a
// hi + lo multiply-add (comp_axpy), as in the other FP32 sweeps.
// DIR as in the one-thread-per-line sweep: 0 the step (Dirichlet ends set
// before and after the solve); 1 ends set before only, raw solution kept;
// 2 ends of the input zeroed, raw solution kept (the adjoint's solves, which
// also read from A.in and write to A.field).
#pragma once

namespace bfvm {
namespace split {

struct SplitArgs {
    int seg;             // elements per segment
    int n_seg;           // segments per line
    const double* sg;    // [s][L] prefix products within segments
    const double* sl;    // [s][L] suffix products within segments
    const float* sg32;   // FP32: [2][s][L] hi then lo
    const float* sl32;
    int64_t n_tab;       // n_sub * L (offset of the lo block)
    void* ex;            // [2][n_seg][n_lines] segment end values
};

// Line `line` of the axis: its first element, stride, substrate, and
// whether it lies entirely on a Dirichlet shell (same numbering and shell
// rules as the one-thread-per-line sweep)
struct SplitLine {
    int64_t base, stride;
    int s;
    bool dir, all_shell;
    double v;
    double v0, v1;   // input values of the two ends (a Dirichlet node's, if one sits there)
};

template <typename T, int AXIS>
__device__ __forceinline__ SplitLine split_line(const SweepArgs<T>& A, int64_t line)
{
    SplitLine L;
    int64_t t = line;
    bool other_shell;
    if (AXIS == 0) {
        const int oy = (int)(t % A.ny); t /= A.ny;
        const int oz = (int)(t % A.nz);
        L.s = (int)(t / A.nz);
        L.base = (((int64_t)L.s * A.nz + oz) * A.ny + oy) * A.pitch;
        L.stride = 1;
        other_shell = (oy == 0 || oy == A.ny - 1 || (((A.zfaces & 1) && oz == 0) || ((A.zfaces & 2) && oz == A.nz - 1)));
    } else if (AXIS == 1) {
        const int ox = (int)(t % A.nx); t /= A.nx;
        const int oz = (int)(t % A.nz);
        L.s = (int)(t / A.nz);
        L.base = (((int64_t)L.s * A.nz + oz) * A.ny) * A.pitch + ox;
        L.stride = A.pitch;
        other_shell = (ox == 0 || ox == A.nx - 1 || (((A.zfaces & 1) && oz == 0) || ((A.zfaces & 2) && oz == A.nz - 1)));
    } else {
        const int ox = (int)(t % A.nx); t /= A.nx;
        const int oy = (int)(t % A.ny);
        L.s = (int)(t / A.ny);
        L.base = ((int64_t)L.s * A.nz * A.ny + oy) * A.pitch + ox;
        L.stride = (int64_t)A.ny * A.pitch;
        other_shell = (ox == 0 || ox == A.nx - 1 || oy == 0 || oy == A.ny - 1);
    }
    L.dir = A.bc_kind[L.s] == BFVM_BC_DIRICHLET;
    L.all_shell = L.dir && other_shell;
    L.v = A.bc_value[L.s];
    end_values(A.ends, line, L.v, L.v0, L.v1);
    return L;
}

// Padded line count of the thread numbering (x lines: whole warps per segment)
template <int AXIS>
__device__ __forceinline__ int64_t split_lines(int64_t n_lines)
{
    return AXIS == 0 ? (n_lines + 31) / 32 * 32 : n_lines;
}

// x lines: copy the warp's 32 rows of elements [k0, k0 + len) between the
// field and the tile ([32][ld] with ld = len + 1); `base` is this lane's row
// base, rows with valid == false are skipped.  Consecutive lanes take
// consecutive elements of a row.
template <typename T, bool LOAD>
__device__ __forceinline__ void tile_copy(T* field, T* tile, int ld, int64_t base, bool valid,
                                          int k0, int len, int lane)
{
    const int total = 32 * len;
    for (int e0 = 0; e0 < total; e0 += 32) {
        const int e = e0 + lane;
        const int row = e / len, k = e - row * len;
        const int64_t rb = __shfl_sync(0xffffffffu, base, row < 32 ? row : 0);
        const int ok = __shfl_sync(0xffffffffu, (int)valid, row < 32 ? row : 0);
        if (e < total && ok) {
            if (LOAD) tile[row * ld + k] = field[rb + k0 + k];
            else field[rb + k0 + k] = tile[row * ld + k];
        }
    }
    __syncwarp();
}

// u * (table entry i) + v: FP64 one FMA; FP32 compensated with the hi + lo
// table (hi block at tab32, lo block n_tab further)
template <typename T>
__device__ __forceinline__ T tab_axpy(const double* tab64, const float* tab32, int64_t n_tab,
                                      int64_t i, T u, T v)
{
    if (sizeof(T) == 8) return (T)fma(tab64[i], (double)u, (double)v);
    return (T)comp_axpy(tab32[i], tab32[n_tab + i], (float)u, (float)v);
}

// Thread t of a pass: segment q and line (x: padding threads of the last
// warp of a segment are inactive and take the last line's geometry).
// Returns false past the last warp.
template <typename T, int AXIS>
__device__ __forceinline__ bool split_thread(const SweepArgs<T>& A, const SplitArgs& Z,
                                             int64_t t, int& q, int64_t& line, bool& active)
{
    const int64_t nl = split_lines<AXIS>(A.n_lines);
    if (t >= nl * Z.n_seg) return false;
    q = (int)(t / nl);
    line = t - (int64_t)q * nl;
    active = line < A.n_lines;
    if (!active) line = A.n_lines - 1;
    return true;
}

// Element k of this thread's segment: the staged tile row (x) or the field
// (read from src, written to f)
template <typename T, int AXIS>
struct SegView {
    T* f;          // output field at the line's base
    const T* src;  // input at the line's base
    int64_t stride;
    T* row;        // tile row of this lane (x)
    int k0;
    __device__ __forceinline__ T get(int k) const
    {
        return AXIS == 0 ? row[k - k0] : src[k * stride];
    }
    __device__ __forceinline__ void put(int k, T v) const
    {
        if (AXIS == 0) row[k - k0] = v;
        else f[k * stride] = v;
    }
};

// 1. forward elimination of each segment from a zero incoming value
template <typename T, int AXIS, int DIR>
__global__ void __launch_bounds__(256) k_split_fwd(SweepArgs<T> A, SplitArgs Z)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int q;
    int64_t line;
    bool active;
    if (!split_thread<T, AXIS>(A, Z, t, q, line, active)) return;
    const SplitLine L = split_line<T, AXIS>(A, line);
    const int n = A.n;
    const int k0 = q * Z.seg, k1 = min(n, k0 + Z.seg);
    const int lane = threadIdx.x & 31, ld = Z.seg + 1;
    T* tile = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * 32 * ld;
    const SegView<T, AXIS> V{A.field + L.base, A.in + L.base, L.stride, tile + lane * ld, k0};
    const double vin = DIR == 2 ? 0.0 : L.v;   // Dirichlet input value
    if (AXIS == 0)
        tile_copy<T, true>(const_cast<T*>(A.in), tile, ld, L.base, active, k0, k1 - k0, lane);
    if (active && L.all_shell && DIR != 1) {
        // the whole line is on the Dirichlet shell: the value, no solve
        for (int k = k0; k < k1; ++k) V.put(k, (T)vin);
    } else if (active) {
        const int64_t row = (int64_t)L.s * A.L + A.axis_off;
        const T c = A.cvec[L.s * 3 + AXIS];
        T prev = (T)0;
        for (int k = k0; k < k1; ++k) {
            T d = V.get(k);
            if (L.all_shell) d = (T)vin;
            else if (L.dir && (k == 0 || k == n - 1))
                d = (T)(DIR != 2 ? (k == 0 ? L.v0 : L.v1) : vin);
            if (sizeof(T) == 8) {
                prev = (T)(fma((double)c, (double)prev, (double)d) * (double)A.r[row + k]);
            } else {
                const float tt = comp_axpy((float)c, (float)A.cvec_lo[L.s * 3 + AXIS],
                                           (float)prev, (float)d);
                prev = (T)__fmaf_rn(tt, (float)A.r[row + k], __fmul_rn(tt, (float)A.r_lo[row + k]));
            }
            V.put(k, prev);
        }
        reinterpret_cast<T*>(Z.ex)[(int64_t)q * A.n_lines + line] = prev;
    }
    if (AXIS == 0) {
        __syncwarp();
        tile_copy<T, false>(A.field, tile, ld, L.base, active, k0, k1 - k0, lane);
    }
}

// 2. incoming d' of each segment, then its back substitution from zero
template <typename T, int AXIS, int DIR>
__global__ void __launch_bounds__(256) k_split_bwd(SweepArgs<T> A, SplitArgs Z)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int q;
    int64_t line;
    bool active;
    if (!split_thread<T, AXIS>(A, Z, t, q, line, active)) return;
    const SplitLine L = split_line<T, AXIS>(A, line);
    const bool solve = active && !(L.all_shell && DIR != 1);   // else written in pass 1
    const int n = A.n;
    const int k0 = q * Z.seg, k1 = min(n, k0 + Z.seg);
    const int lane = threadIdx.x & 31, ld = Z.seg + 1;
    T* tile = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * 32 * ld;
    const SegView<T, AXIS> V{A.field + L.base, A.field + L.base, L.stride, tile + lane * ld, k0};
    if (AXIS == 0) tile_copy<T, true>(A.field, tile, ld, L.base, solve, k0, k1 - k0, lane);
    if (solve) {
        const int64_t row = (int64_t)L.s * A.L + A.axis_off;
        const T* exA = reinterpret_cast<const T*>(Z.ex);
        T* exC = reinterpret_cast<T*>(Z.ex) + A.n_lines * Z.n_seg;
        // D_j = f_last(j) + G(last of j) D_{j-1}, from D_{-1} = 0
        T D = (T)0;
        for (int j = 0; j < q; ++j) {
            const int last = min(n, (j + 1) * Z.seg) - 1;
            D = tab_axpy<T>(Z.sg, Z.sg32, Z.n_tab, row + last, D, exA[(int64_t)j * A.n_lines + line]);
        }
        T x = (T)0;
        for (int k = k1 - 1; k >= k0; --k) {
            const T dp = tab_axpy<T>(Z.sg, Z.sg32, Z.n_tab, row + k, D, V.get(k));
            if (sizeof(T) == 8)
                x = (T)fma((double)A.cr[row + k], (double)x, (double)dp);
            else
                x = (T)comp_axpy((float)A.cr[row + k], (float)A.cr_lo[row + k], (float)x, (float)dp);
            V.put(k, x);
        }
        exC[(int64_t)q * A.n_lines + line] = x;
    }
    if (AXIS == 0) {
        __syncwarp();
        tile_copy<T, false>(A.field, tile, ld, L.base, solve, k0, k1 - k0, lane);
    }
}

// 3. incoming x of each segment, the solution, and the Dirichlet ends
template <typename T, int AXIS, int DIR>
__global__ void __launch_bounds__(256) k_split_out(SweepArgs<T> A, SplitArgs Z)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int q;
    int64_t line;
    bool active;
    if (!split_thread<T, AXIS>(A, Z, t, q, line, active)) return;
    const SplitLine L = split_line<T, AXIS>(A, line);
    const bool solve = active && !(L.all_shell && DIR != 1);
    const int n = A.n;
    const int k0 = q * Z.seg, k1 = min(n, k0 + Z.seg);
    const int lane = threadIdx.x & 31, ld = Z.seg + 1;
    T* tile = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * 32 * ld;
    const SegView<T, AXIS> V{A.field + L.base, A.field + L.base, L.stride, tile + lane * ld, k0};
    if (AXIS == 0) tile_copy<T, true>(A.field, tile, ld, L.base, solve, k0, k1 - k0, lane);
    if (solve) {
        const int64_t row = (int64_t)L.s * A.L + A.axis_off;
        const T* exC = reinterpret_cast<const T*>(Z.ex) + A.n_lines * Z.n_seg;
        // X_j = g_first(j) + S(first of j) X_{j+1}, from X_{n_seg} = 0
        T X = (T)0;
        for (int j = Z.n_seg - 1; j > q; --j)
            X = tab_axpy<T>(Z.sl, Z.sl32, Z.n_tab, row + (int64_t)j * Z.seg, X,
                            exC[(int64_t)j * A.n_lines + line]);
        for (int k = k0; k < k1; ++k) {
            T x = tab_axpy<T>(Z.sl, Z.sl32, Z.n_tab, row + k, X, V.get(k));
            if (DIR == 0 && L.dir && (k == 0 || k == n - 1)) x = (T)L.v;
            V.put(k, x);
        }
    }
    if (AXIS == 0) {
        __syncwarp();
        tile_copy<T, false>(A.field, tile, ld, L.base, solve, k0, k1 - k0, lane);
    }
}

}  // namespace split
}  // namespace bfvm
