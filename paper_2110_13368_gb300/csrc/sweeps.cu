// LOD line sweeps (the x-, y- and z-diffusion of the paper's "Using OpenACC
// programming model for PhysiCell", one implicit tridiagonal solve per line)
// with the Dirichlet condition of "Elements of Parallelism" fused in.
//
// Work decomposition: one thread per line, one warp per 32 consecutive
// lines of a flattened line index (substrate-major, then the two other
// coordinates with x fastest for the y and z sweeps).  For the y and z
// sweeps adjacent lanes therefore touch adjacent x, so every per-element
// access of a warp is one coalesced row.  Each thread copies its whole line
// into a private column of shared memory with cp.async before solving, so
// the line is read from HBM once and written once; the forward elimination
// runs in place in shared memory and the back substitution writes the
// result straight to the field.
//
// Lines too long for shared memory fall back to keeping the forward
// intermediates in the field itself (the field is overwritten in place).
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bfvm {

namespace {

constexpr int kGroups = 8;   // cp.async commit groups per line

__device__ __forceinline__ void cp_async_elem(double* dst, const double* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(float* dst, const float* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
// 16 bytes, both addresses 16-byte aligned; not cached in L1
__device__ __forceinline__ void cp_async_16(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// wait until at most `pending` of this thread's newest groups are in flight
__device__ __forceinline__ void cp_async_wait_dyn(int pending)
{
    switch (pending) {
        case 0: cp_async_wait<0>(); break;
        case 1: cp_async_wait<1>(); break;
        case 2: cp_async_wait<2>(); break;
        case 3: cp_async_wait<3>(); break;
        case 4: cp_async_wait<4>(); break;
        case 5: cp_async_wait<5>(); break;
        case 6: cp_async_wait<6>(); break;
        default: cp_async_wait<7>(); break;
    }
}

template <typename T>
struct SweepArgs {
    const T* in;           // field read (may equal out)
    T* field;              // field written
    int64_t pitch;
    int nx, ny, nz, n_sub;
    int n;                 // line length (extent of the swept axis)
    int64_t n_lines;       // n_sub * (product of the two other extents)
    int64_t L;             // coefficient row length nx + ny + nz
    int axis_off;          // offset of this axis in a coefficient row
    int off_x, off_y, off_z;
    // plain form
    const T* r;            // [s][L] 1/den
    const T* cr;           // [s][L] c/den
    const T* cvec;         // [s][3]
    // FP32 form: low parts of the hi + lo coefficient pairs (null for FP64)
    const T* r_lo;
    const T* cr_lo;
    const T* cvec_lo;
    // rescaled form (FP64): state p tables
    const double* fa;      // [s][L]
    const double* fb;
    const double* sc_p;    // [s][L] scales of state p
    const double* sc_p1;   // [s][L] scales of state p + 1
    const double* isc_p1;  // [s][L] inverses of state p + 1
    const int32_t* bc_kind;
    const double* bc_value;
    int dims;              // 3, or 2: the single z layer of a 2-D grid is not a boundary
    int zfaces;            // z planes on the grid's boundary: bit 0 z = 0, bit 1 z = nz - 1
    T* field2;             // second copy of the output (per-axis pair kernel with DUAL)
    // Dirichlet nodes at line ends: [line][2] raw node values at the k = 0
    // and k = n - 1 ends of each line of a Dirichlet substrate (NaN where no
    // node sits), lines numbered as by full_line; null when no node lies on
    // a Dirichlet shell face
    const double* ends;
};

// Line number of the line along AXIS through (ox, oy, oz) of substrate s, over
// all lines of the grid (the one-thread-per-line sweep's numbering)
template <typename T, int AXIS>
__device__ __forceinline__ int64_t full_line(const SweepArgs<T>& A, int s, int ox, int oy, int oz)
{
    if (AXIS == 0) return ((int64_t)s * A.nz + oz) * A.ny + oy;
    if (AXIS == 1) return ((int64_t)s * A.nz + oz) * A.nx + ox;
    return ((int64_t)s * A.ny + oy) * A.nx + ox;
}

// Unscaled input values of the two ends of a Dirichlet line: the boundary
// value v, or the value of a Dirichlet node sitting at that end (the node is
// applied right after the shell, so the solve sees the node's value there)
__device__ __forceinline__ void end_values(const double* ends, int64_t fl, double v, double& v0,
                                           double& v1)
{
    v0 = v;
    v1 = v;
    if (ends) {
        const double e0 = ends[2 * fl], e1 = ends[2 * fl + 1];
        if (!isnan(e0)) v0 = e0;
        if (!isnan(e1)) v1 = e1;
    }
}

// MODE 0: plain Thomas (3 flops per element: FMA + MUL forward, FMA back).
// MODE 1: rescaled Thomas (one FMA forward, one FMA back).
// MODE 2: rescaled, and the z sweep divides the accumulated scale out.
// DIR 0: Dirichlet shell set before and after the solve (the step itself).
// DIR 1: shell set before the solve only; the raw solution is kept (the
//        replay of a step for the adjoint needs it).
// DIR 2: shell of the input zeroed, raw solution kept (the adjoint solve:
//        the Dirichlet projection's Jacobian is zero on the shell).
// a*u + v for an FP32 coefficient held as a = hi + lo (lo the rounding error
// of hi), as fl(fl(hi*u + fl(lo*u)) + v): the low part's product enters the
// FMA below its rounding, so the product is rounded once from a*u itself
// and carries no bias from the coefficient's own rounding (which would push
// every sweep the same way); the sum then rounds once more.  Both roundings
// are to nearest; in the Thomas recurrences every term is non-negative for a
// non-negative field, so nothing cancels.  Three operations, three deep on
// the recurrence's chain (a TwoSum-compensated sum, one rounding in all,
// took eleven, nine deep, on chains that bound the FP32 sweeps).  Explicit
// _rn intrinsics keep the compiler from contracting them.
__device__ __forceinline__ float comp_axpy(float a_hi, float a_lo, float u, float v)
{
    return __fadd_rn(__fmaf_rn(a_hi, u, __fmul_rn(a_lo, u)), v);
}

// One line per thread: the generic sweep used by the adjoint passes, by the
// batched form and for lines too long for the persistent kernel.  `wsm` is
// this warp's shared column buffer (32 x n elements) when SMEM.
template <typename T, int AXIS, int MODE, int DIR, bool SMEM>
__device__ __forceinline__ void sweep_one_line(const SweepArgs<T>& A, int64_t line, int lane,
                                               T* wsm)
{

    const int n = A.n;
    int s, ox, oy, oz;   // substrate and the two fixed coordinates (third = -1)
    int64_t base, stride;
    bool other_shell;
    if (AXIS == 0) {
        int64_t t = line;
        oy = (int)(t % A.ny); t /= A.ny;
        oz = (int)(t % A.nz); s = (int)(t / A.nz);
        ox = -1;
        base = (((int64_t)s * A.nz + oz) * A.ny + oy) * A.pitch;
        stride = 1;
        other_shell = (oy == 0 || oy == A.ny - 1 || (((A.zfaces & 1) && oz == 0) || ((A.zfaces & 2) && oz == A.nz - 1)));
    } else if (AXIS == 1) {
        int64_t t = line;
        ox = (int)(t % A.nx); t /= A.nx;
        oz = (int)(t % A.nz); s = (int)(t / A.nz);
        oy = -1;
        base = (((int64_t)s * A.nz + oz) * A.ny) * A.pitch + ox;
        stride = A.pitch;
        other_shell = (ox == 0 || ox == A.nx - 1 || (((A.zfaces & 1) && oz == 0) || ((A.zfaces & 2) && oz == A.nz - 1)));
    } else {
        int64_t t = line;
        ox = (int)(t % A.nx); t /= A.nx;
        oy = (int)(t % A.ny); s = (int)(t / A.ny);
        oz = -1;
        base = ((int64_t)s * A.nz * A.ny + oy) * A.pitch + ox;
        stride = (int64_t)A.ny * A.pitch;
        other_shell = (ox == 0 || ox == A.nx - 1 || oy == 0 || oy == A.ny - 1);
    }
    const bool dir = A.bc_kind[s] == BFVM_BC_DIRICHLET;
    const double v = (DIR == 2) ? 0.0 : A.bc_value[s];
    const T* fin = A.in + base;
    T* f = A.field + base;
    const int64_t row = (int64_t)s * A.L;

    // Scale bookkeeping of the rescaled form.  At the sweep of AXIS in state
    // p the axes before it are already in state p + 1, the others in p.
    double kline = 1.0;      // Dirichlet value times the other axes' scales
    double inv_other = 1.0;  // inverse of the other axes' scales (MODE 2)
    const double* own_in = nullptr;
    const double* own_out = nullptr;
    // the two ends' input values (a Dirichlet node may sit at either end;
    // the adjoint's solve zeroes them like the shell)
    double v0 = v, v1 = v;
    if (DIR != 2) end_values(A.ends, line, v, v0, v1);
    double kl0 = v0, kl1 = v1;
    if (MODE >= 1) {
        own_in = A.sc_p + row + A.axis_off;
        own_out = A.sc_p1 + row + A.axis_off;
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
            if (MODE == 2)
                inv_other = A.isc_p1[row + A.off_x + ox] * A.isc_p1[row + A.off_y + oy];
        }
        kline = v * sa * sb;
        kl0 = v0 * sa * sb;
        kl1 = v1 * sa * sb;
    }

    if (dir && other_shell && DIR != 1) {
        // the whole line is on the Dirichlet shell: no solve, just the value
        // (the adjoint's zeroed input solves to zero)
        for (int k = 0; k < n; ++k) {
            double val;
            if (MODE == 0 || MODE == 2) val = v;
            else val = kline * own_out[k];
            f[k * stride] = (T)val;
        }
        return;
    }

    T* w;
    int64_t wstride;
    if (SMEM) {
        w = wsm + lane;
        wstride = 32;
        const int gs = (n + kGroups - 1) / kGroups;
        for (int g = 0; g < kGroups; ++g) {
            int k0 = g * gs, k1 = min(n, k0 + gs);
            for (int k = k0; k < k1; ++k) cp_async_elem(w + k * 32, fin + k * stride);
            cp_async_commit();
        }
    } else {
        // forward intermediates kept in the output field itself
        w = f;
        wstride = stride;
        if (A.in != A.field)
            for (int k = 0; k < n; ++k) f[k * stride] = fin[k * stride];
    }
    // on a Dirichlet shell line every input element is the shell value
    const bool all_in = dir && other_shell;

    // Dirichlet prologue value of the two line ends (and of a shell line)
    auto end_in = [&](int k) -> T {
        if (MODE == 0) return (T)(all_in ? v : (k == 0 ? v0 : v1));
        return (T)((all_in ? kline : (k == 0 ? kl0 : kl1)) * own_in[k]);
    };

    // forward elimination (in place)
    T prev = (T)0;
    if (MODE == 0 && sizeof(T) == 8) {
        const T c = A.cvec[s * 3 + AXIS];
        const T* __restrict__ r = A.r + row + A.axis_off;
        const int gs = (n + kGroups - 1) / kGroups;
        for (int g = 0; g < kGroups; ++g) {
            if (SMEM) cp_async_wait_dyn(kGroups - 1 - g);
            int k0 = g * gs, k1 = min(n, k0 + gs);
            for (int k = k0; k < k1; ++k) {
                T d = w[k * wstride];
                if (all_in || (dir && (k == 0 || k == n - 1))) d = end_in(k);
                prev = fma(c, prev, d) * r[k];
                w[k * wstride] = prev;
            }
        }
    } else if (MODE == 0) {
        // FP32: coefficients as hi + lo pairs
        const T c = A.cvec[s * 3 + AXIS];
        const T c_lo = A.cvec_lo[s * 3 + AXIS];
        const T* __restrict__ r = A.r + row + A.axis_off;
        const T* __restrict__ r_lo = A.r_lo + row + A.axis_off;
        const int gs = (n + kGroups - 1) / kGroups;
        for (int g = 0; g < kGroups; ++g) {
            if (SMEM) cp_async_wait_dyn(kGroups - 1 - g);
            int k0 = g * gs, k1 = min(n, k0 + gs);
            for (int k = k0; k < k1; ++k) {
                T d = w[k * wstride];
                if (all_in || (dir && (k == 0 || k == n - 1))) d = end_in(k);
                float t = comp_axpy((float)c, (float)c_lo, (float)prev, (float)d);
                prev = (T)__fmaf_rn(t, (float)r[k], __fmul_rn(t, (float)r_lo[k]));
                w[k * wstride] = prev;
            }
        }
    } else {
        const double* __restrict__ fa = A.fa + row + A.axis_off;
        const int gs = (n + kGroups - 1) / kGroups;
        for (int g = 0; g < kGroups; ++g) {
            if (SMEM) cp_async_wait_dyn(kGroups - 1 - g);
            int k0 = g * gs, k1 = min(n, k0 + gs);
            for (int k = k0; k < k1; ++k) {
                T d = w[k * wstride];
                if (all_in || (dir && (k == 0 || k == n - 1))) d = end_in(k);
                prev = fma((T)fa[k], prev, d);
                w[k * wstride] = prev;
            }
        }
    }

    // back substitution, result written to the field
    auto emit = [&](int k, T x) {
        T out;
        if (DIR == 0 && dir && (k == 0 || k == n - 1)) {
            if (MODE == 0 || MODE == 2) out = (T)v;
            else out = (T)(kline * own_out[k]);
        } else if (MODE == 2) {
            out = (T)((x * A.isc_p1[row + A.axis_off + k]) * inv_other);
        } else {
            out = x;
        }
        f[k * stride] = out;
    };
    T x = prev;
    emit(n - 1, x);
    if (MODE == 0 && sizeof(T) == 8) {
        const T* __restrict__ cr = A.cr + row + A.axis_off;
        for (int k = n - 2; k >= 0; --k) {
            x = fma(cr[k], x, w[k * wstride]);
            emit(k, x);
        }
    } else if (MODE == 0) {
        const T* __restrict__ cr = A.cr + row + A.axis_off;
        const T* __restrict__ cr_lo = A.cr_lo + row + A.axis_off;
        for (int k = n - 2; k >= 0; --k) {
            x = (T)comp_axpy((float)cr[k], (float)cr_lo[k], (float)x, (float)w[k * wstride]);
            emit(k, x);
        }
    } else {
        const double* __restrict__ fb = A.fb + row + A.axis_off;
        for (int k = n - 2; k >= 0; --k) {
            x = fma((T)fb[k], x, w[k * wstride]);
            emit(k, x);
        }
    }
}

template <typename T, int AXIS, int MODE, int DIR, bool SMEM>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= A.n_lines) return;
    T* wsm = SMEM ? reinterpret_cast<T*>(smem_raw) + (int64_t)warp * 32 * A.n : nullptr;
    sweep_one_line<T, AXIS, MODE, DIR, SMEM>(A, line, lane, wsm);
}

// rho <- alpha rho + beta over the occupied voxels (cell sources and sinks,
// the delta term of Eq. 1, with every voxel's cells composed in index order).
// In the rescaled form the field carries the scale X(x) Y(y) Z(z) of the
// current state, so beta is scaled alike.
template <typename T, bool SCALED>
__global__ void k_sources(T* __restrict__ field, int64_t n_entries, const int64_t* count,
                          const int64_t* __restrict__ off,
                          const double* __restrict__ alpha,
                          const double* __restrict__ beta,
                          const int32_t* __restrict__ vox,
                          const int32_t* __restrict__ sub, int nx, int ny,
                          int64_t L, int off_y, int off_z,
                          const double* __restrict__ sc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (count) n_entries = count[1];   // tables re-binned on the device since the host counted
    if (e >= n_entries) return;
    int64_t o = off[e];
    double b = beta[e];
    if (SCALED) {
        int32_t vv = vox[e];
        int x = vv % nx;
        int y = (vv / nx) % ny;
        int z = vv / (nx * ny);
        const double* t = sc + (int64_t)sub[e] * L;
        b *= t[x] * t[off_y + y] * t[off_z + z];
    }
    double r = (double)field[o];
    field[o] = (T)fma(alpha[e], r, b);
}

}  // namespace
}  // namespace bfvm

#include "sweep_persistent.cuh"
#include "sweep_pair.cuh"
#include "sweep_step.cuh"
#include "sweep_batch_step.cuh"
#include "sweep_split.cuh"

namespace bfvm {
namespace {

template <typename T>
SweepArgs<T> make_args(Ctx* c, int axis, int p, const T* r, const T* cr,
                       const T* cvec)
{
    SweepArgs<T> A{};
    A.field = reinterpret_cast<T*>(c->field);
    A.in = A.field;
    A.pitch = c->pitch;
    A.nx = c->nx; A.ny = c->ny; A.nz = c->nz; A.n_sub = c->n_sub;
    int ext[3] = {c->nx, c->ny, c->nz};
    A.n = ext[axis];
    int64_t other = (int64_t)ext[0] * ext[1] * ext[2] / ext[axis];
    A.n_lines = other * c->n_sub;
    A.L = c->coef.L;
    A.off_x = 0; A.off_y = c->nx; A.off_z = c->nx + c->ny;
    A.axis_off = axis == 0 ? 0 : (axis == 1 ? A.off_y : A.off_z);
    A.r = r; A.cr = cr; A.cvec = cvec;
    if (sizeof(T) == 4) {
        int64_t n_tab = (int64_t)c->n_sub * c->coef.L;
        A.r_lo = r + n_tab;
        A.cr_lo = cr + n_tab;
        A.cvec_lo = cvec + (int64_t)c->n_sub * 3;
    }
    if (c->coef.fa) {
        int64_t per_state = (int64_t)c->n_sub * c->coef.L;
        A.fa = c->coef.fa + (int64_t)p * per_state;
        A.fb = c->coef.fb + (int64_t)p * per_state;
        A.sc_p = c->coef.sc + (int64_t)p * per_state;
        A.sc_p1 = c->coef.sc + (int64_t)(p + 1) * per_state;
        A.isc_p1 = c->coef.isc + (int64_t)(p + 1) * per_state;
    }
    A.bc_kind = c->d_bc_kind;
    A.bc_value = c->d_bc_value;
    A.dims = c->dims;
    A.zfaces = c->zfaces();
    A.ends = c->d_node_ends[axis];
    return A;
}

// The split line solve of one axis (sweep_split.cuh): three launches.
template <typename T, int AXIS, int DIR>
bfvm_status launch_split(Ctx* c, const SweepArgs<T>& A)
{
    split::SplitArgs Z;
    Z.seg = c->coef.seg[AXIS];
    if (Z.seg < 1 || !c->coef.split_ex) return set_err(c, BFVM_ESTATE, "split tables missing");
    Z.n_seg = (int)ceil_div(A.n, Z.seg);
    Z.sg = c->coef.sg;
    Z.sl = c->coef.sl;
    Z.sg32 = c->coef.sg32;
    Z.sl32 = c->coef.sl32;
    Z.n_tab = (int64_t)c->n_sub * c->coef.L;
    Z.ex = c->coef.split_ex;
    if (A.n_lines == 0) return BFVM_OK;
    // x lines: whole warps per segment and a staging tile of 32 x (seg + 1)
    // elements per warp (seg <= 64, so at least 2 warps fit in 48 KB)
    const int64_t lines = AXIS == 0 ? ceil_div(A.n_lines, 32) * 32 : A.n_lines;
    const int64_t nt = lines * Z.n_seg;
    int block = 256;
    size_t smem = 0;
    if (AXIS == 0) {
        const size_t tile = (size_t)32 * (Z.seg + 1) * sizeof(T);
        const int warps = (int)std::min<size_t>(8, std::max<size_t>(1, (48 << 10) / tile));
        block = 32 * warps;
        smem = tile * warps;
    }
    const unsigned grid = (unsigned)ceil_div(nt, block);
    split::k_split_fwd<T, AXIS, DIR><<<grid, block, smem, c->stream>>>(A, Z);
    split::k_split_bwd<T, AXIS, DIR><<<grid, block, smem, c->stream>>>(A, Z);
    split::k_split_out<T, AXIS, DIR><<<grid, block, smem, c->stream>>>(A, Z);
    c->launches += 3;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

template <typename T, int AXIS, int MODE, int DIR = 0>
bfvm_status launch_axis(Ctx* c, const SweepArgs<T>& A)
{
    constexpr int G = persistent::Groups<T>::G;
    const int ns = (int)ceil_div(A.n, G) * G;
    const size_t per_warp = (size_t)32 * ns * sizeof(T) + 2 * 32 * sizeof(int64_t);
    const int ncoef = (MODE == 0 ? (sizeof(T) == 4 ? 4 : 2) : 2);
    size_t fixed = (((size_t)A.n_sub * ncoef * A.n * sizeof(T) + 15) & ~(size_t)15) +
                   (MODE == 2 ? (((size_t)A.n_sub * A.n * 8 + 15) & ~(size_t)15) : 0) +
                   ((((size_t)A.n_sub + 1) * 8 + 15) & ~(size_t)15);
    int max_warps = sizeof(T) == 8 ? 4 : 8;
    int warps = 0;
    // the shared-memory sweeps run the step's Dirichlet handling; the
    // adjoint's solves (DIR 1, 2) differ from it only on Dirichlet
    // substrates, so without those they take the same kernels
    bool any_dir = false;
    for (int s = 0; s < c->n_sub; ++s) any_dir = any_dir || c->bc_kind[s] == BFVM_BC_DIRICHLET;
    if ((DIR == 0 || !any_dir) && A.n_sub <= 64 && c->smem_optin > fixed)
        warps = (int)((c->smem_optin - fixed) / per_warp);
    if (warps > max_warps) warps = max_warps;
    KernelTimer timer(c, AXIS);
    // plain-form sweeps: the split solve where one thread or one 32-line
    // block per line cannot fill the GPU (the 2-D variant) or the step's
    // lines are too long for the shared-memory kernels; the adjoint's solves
    // (DIR 1, 2) only when forced (on the 100^3 adjoint workload it gained
    // nothing over one thread per line)
    if (MODE == 0 &&
        (c->split == 2 || (c->split == 1 && DIR == 0 && (c->dims == 2 || warps < 1))))
        return launch_split<T, AXIS, DIR>(c, A);
    if (warps >= 1) {
        const int64_t* first = c->lines_first[AXIS];
        if (first[A.n_sub] == 0) return BFVM_OK;   // every line is on the shell
        if (!c->line_tables_ready[AXIS]) return set_err(c, BFVM_ESTATE, "line tables missing");
        persistent::LineSet S;
        S.n_sub = A.n_sub;
        S.first = c->d_first[AXIS];
        S.lo_a = c->d_lo_a[AXIS];
        S.cnt_a = c->d_cnt_a[AXIS];
        S.lo_b = c->d_lo_b[AXIS];
        // one column buffer per warp pair (see sweep_pair.cuh)
        const size_t per_pair = (size_t)32 * ns * sizeof(T) + 4 * 32 * sizeof(int64_t) +
                                32 * sizeof(T);
        int pairs = (int)((c->smem_optin - fixed) / per_pair);
        if (pairs > persistent::Groups<T>::AXIS_PAIRS) pairs = persistent::Groups<T>::AXIS_PAIRS;
        if (c->sweep_kernel == 0 && pairs >= 1) {
            const int64_t n_blocks = ceil_div(first[A.n_sub], 32);
            // spread the pairs over every SM where there are few blocks (a
            // 100^3 grid has 313 per axis: 3 pairs per CTA on 105 SMs rather
            // than 4 on 79; the 100^3 adjoint backward 36.9 -> 36.6 ms)
            const int64_t per_sm = ceil_div(n_blocks, (int64_t)c->sm_count);
            if (per_sm < pairs) pairs = (int)(per_sm > 1 ? per_sm : 1);
            size_t smem = fixed + per_pair * pairs;
            auto kern = persistent::k_sweep_pair<T, AXIS, MODE>;
            if constexpr (sizeof(T) == 8 && MODE == 0) {
                if (A.field2) {   // the adjoint's replay: a second copy of the output
                    kern = persistent::k_sweep_pair<T, AXIS, MODE, true>;
                    c->dual_done = true;
                }
            }
            BFVM_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
            int64_t grid = ceil_div(n_blocks, pairs);
            if (grid > c->sm_count) grid = c->sm_count;
            if (c->grid_limit > 0 && grid > c->grid_limit) grid = c->grid_limit;
            kern<<<(unsigned)grid, 64 * pairs, smem, c->stream>>>(A, S, n_blocks, ns);
            c->launches += 1;
            BFVM_CUDA(c, cudaGetLastError());
            return BFVM_OK;
        }
        size_t smem = fixed + per_warp * warps;
        auto kern = persistent::k_sweep_persistent<T, AXIS, MODE>;
        BFVM_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        int64_t n_blocks = ceil_div(first[A.n_sub], 32);
        int64_t grid = ceil_div(n_blocks, warps);
        if (grid > c->sm_count) grid = c->sm_count;
        if (c->grid_limit > 0 && grid > c->grid_limit) grid = c->grid_limit;
        kern<<<(unsigned)grid, 32 * warps, smem, c->stream>>>(A, S, n_blocks, ns);
    } else {
        size_t per_warp1 = (size_t)32 * A.n * sizeof(T);
        int w1 = (int)(c->smem_optin / per_warp1);
        if (w1 > 4) w1 = 4;
        if (w1 >= 1) {
            // generic form (adjoint passes): one warp per 32 lines, lines
            // staged in shared memory
            size_t smem = per_warp1 * w1;
            auto kern = k_sweep<T, AXIS, MODE, DIR, true>;
            BFVM_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
            kern<<<(unsigned)ceil_div(A.n_lines, 32 * w1), 32 * w1, smem, c->stream>>>(A);
        } else {
            // lines too long for shared memory: intermediates kept in the field
            auto kern = k_sweep<T, AXIS, MODE, DIR, false>;
            kern<<<(unsigned)ceil_div(A.n_lines, 128), 128, 0, c->stream>>>(A);
        }
    }
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

// The x, y and z sweeps of a step as one persistent launch (sweep_step.cuh):
// the rescaled FP64 form (MXY 1), the plain FP64 form and the FP32 form
// (MXY 0).  Returns BFVM_ESTATE without launching when the context does not
// qualify (the caller then launches the axes one by one).
bfvm_status launch_nodes(Ctx* c, int p, bool renorm, int stage);

template <typename T, int MXY>
bfvm_status launch_step_fused(Ctx* c, int p, bool renorm, const T* r, const T* cr,
                              const T* cvec)
{
    // also runs the step's Dirichlet shell and cell sources (its epilogue)
    constexpr int G = persistent::Groups<T>::G;
    constexpr int NC = persistent::step_ncoef<T, MXY>();
    // Dirichlet nodes: FP64 only, with the node tables built for this task list
    const bool nodes = c->n_nodes > 0;
    if (!c->fused_step || c->sweep_kernel != 0 || !c->d_task_first || !c->d_sched ||
        c->n_sub > 64 || c->dims != 3 || (nodes && (sizeof(T) != 8 || !c->d_node_task_first)))
        return BFVM_ESTATE;
    for (int a = 0; a < 3; ++a)
        if (!c->line_tables_ready[a]) return BFVM_ESTATE;
    const int ext[3] = {c->nx, c->ny, c->nz};
    int ns = 0;
    for (int a = 0; a < 3; ++a) ns = std::max(ns, (int)ceil_div(ext[a], G) * G);
    const persistent::StepSmem M = persistent::step_smem<T>(c->n_sub, c->coef.L, NC, ns);
    if (c->smem_optin < M.fixed + M.pair) return BFVM_ESTATE;
    constexpr int MAXP = persistent::Groups<T>::MAX_PAIRS;
    int pairs = (int)((c->smem_optin - M.fixed) / M.pair);
    if (pairs > MAXP) pairs = MAXP;
    // the per-axis launches stage one axis' coefficients only; where that
    // leaves room for more pairs, they are the faster choice
    const size_t fixed_axis = (size_t)c->n_sub * NC * ns * sizeof(T) + 1024;
    const int pairs_axis = (int)std::min<size_t>(persistent::Groups<T>::AXIS_PAIRS,
                                                 (c->smem_optin - fixed_axis) / M.pair);
    if (c->fused_step != 2) {
        if (pairs < pairs_axis) return BFVM_ESTATE;
        // FP32: the per-axis launches measured faster at equal pair counts
        // (200^3 step 0.166 ms against 0.194 ms in one launch)
        if (sizeof(T) == 4) return BFVM_ESTATE;
    }
    // the node values the x sweep reads (the shell's part is the line ends)
    if (nodes) {
        const bfvm_status st = launch_nodes(c, p, renorm, 0);
        if (st != BFVM_OK) return st;
    }
    KernelTimer timer(c, 4);
    SweepArgs<T> A[3];
    persistent::LineSet S[3];
    for (int a = 0; a < 3; ++a) {
        A[a] = make_args<T>(c, a, p, r, cr, cvec);
        S[a].n_sub = c->n_sub;
        S[a].first = c->d_first[a];
        S[a].lo_a = c->d_lo_a[a];
        S[a].cnt_a = c->d_cnt_a[a];
        S[a].lo_b = c->d_lo_b[a];
    }
    persistent::StepSched Q;
    Q.claim = c->d_sched;
    Q.exit_count = c->d_sched + 1;
    Q.done = c->d_sched + 2;
    Q.task_first = c->d_task_first;
    Q.err = c->d_err + 1;
    Q.n_sub = c->n_sub;
    Q.n_tasks = c->n_tasks;
    Q.max_polls = c->wait_test_polls > 0 ? (unsigned)c->wait_test_polls : persistent::kMaxPolls;
    Q.extra_need = c->wait_test_polls > 0 ? 1u : 0u;
    Q.eclaim = c->d_sched + 2 + 3 * c->n_sub;
    Q.shell_done = Q.eclaim + 1;
    // occupied voxels: exact, or (after a device-only cell update) the
    // capacity, with the exact count read by the kernel
    const int64_t n_seg = c->src.counts_on_host ? c->src.n_seg : c->src.cap;
    int64_t n_epi = 0;
    for (int s = 0; s < c->n_sub; ++s)
        n_epi += (c->bc_kind[s] == BFVM_BC_DIRICHLET ? persistent::epi_shell_chunks(c->nx, c->ny, c->nz) : 0) +
                 (nodes ? c->node_chunks[s] : 0) + persistent::epi_src_chunks(n_seg);
    Q.n_epi_chunks = (int)n_epi;
    Q.node_task_first = nodes ? c->d_node_task_first : nullptr;
    Q.node_patch = nodes ? c->d_node_patch : nullptr;
    Q.node_sfirst = nodes ? c->d_node_sfirst : nullptr;
    Q.node_epi = nodes ? c->d_node_epi : nullptr;
    persistent::EpiArgs<T> E;
    E.field = reinterpret_cast<T*>(c->field);
    E.nx = c->nx;
    E.ny = c->ny;
    E.nz = c->nz;
    E.pitch = c->pitch;
    E.L = c->coef.L;
    E.sc = (MXY == 0 || renorm) ? nullptr : A[0].sc_p1;
    E.n_seg = n_seg;
    E.d_nseg = c->src.counts_on_host ? nullptr : c->src.d_count;
    E.off = c->src.off;
    E.alpha = c->src.alpha;
    E.beta = c->src.beta;
    E.vox = c->src.vox;
    E.sub = c->src.sub;
    E.zf = c->zfaces();
    const size_t smem = M.fixed + M.pair * pairs;
    int64_t grid = ceil_div(std::max<int64_t>(c->n_tasks, 1), pairs);
    grid = std::max<int64_t>(grid, ceil_div(Q.n_epi_chunks, 8 * pairs));
    if (grid > c->sm_count) grid = c->sm_count;
    if (c->grid_limit > 0 && grid > c->grid_limit) grid = c->grid_limit;
    auto kern = persistent::k_step_pair<T, MXY, MXY, false>;
    if (MXY == 1 && renorm) kern = persistent::k_step_pair<T, MXY, 2 * MXY, false>;
    if constexpr (sizeof(T) == 8) {
        if (nodes) {
            kern = persistent::k_step_pair<T, MXY, MXY, true>;
            if (MXY == 1 && renorm) kern = persistent::k_step_pair<T, MXY, 2 * MXY, true>;
        }
    }
    BFVM_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    kern<<<(unsigned)grid, 64 * pairs, smem, c->stream>>>(A[0], A[1], A[2], S[0], S[1], S[2], Q,
                                                          E, ns);
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

// Dirichlet nodes inside the domain: field <- value at each node, times the
// scales the field carries at that point of a rescaled step (the axes
// already swept in state p + 1, the others in state p; plain values after a
// renormalising z sweep and in the plain forms).
template <typename T>
__global__ void k_nodes(T* __restrict__ field, int64_t n, const int64_t* __restrict__ off,
                        const int32_t* __restrict__ vox, const int32_t* __restrict__ sub,
                        const double* __restrict__ val, int nx, int ny, int64_t L,
                        const double* __restrict__ sx, const double* __restrict__ sy,
                        const double* __restrict__ sz)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double v = val[e];
    if (sx) {
        const int32_t vv = vox[e];
        const int x = vv % nx, y = (vv / nx) % ny, z = vv / (nx * ny);
        const int64_t row = (int64_t)sub[e] * L;
        v = v * (sx[row + x] * sy[row + nx + y] * sz[row + nx + ny + z]);
    }
    field[off[e]] = (T)v;
}

// stage 0: before the x sweep, 1: after x, 2: after y, 3: after z and the
// Dirichlet shell
bfvm_status launch_nodes(Ctx* c, int p, bool renorm, int stage)
{
    if (c->n_nodes == 0) return BFVM_OK;
    const double *sx = nullptr, *sy = nullptr, *sz = nullptr;
    if (c->precision == 64 && c->variant == 1 && !(renorm && stage == 3)) {
        const int64_t per = (int64_t)c->n_sub * c->coef.L;
        const double* s0 = c->coef.sc + (int64_t)p * per;
        const double* s1 = c->coef.sc + (int64_t)(p + 1) * per;
        sx = stage >= 1 ? s1 : s0;
        sy = stage >= 2 ? s1 : s0;
        sz = stage >= 3 ? s1 : s0;
    }
    KernelTimer timer(c, 3);
    const unsigned grid = (unsigned)ceil_div(c->n_nodes, 256);
    if (c->precision == 64)
        k_nodes<double><<<grid, 256, 0, c->stream>>>(
            reinterpret_cast<double*>(c->field), c->n_nodes, c->d_node_off, c->d_node_vox,
            c->d_node_sub, c->d_node_val, c->nx, c->ny, c->coef.L, sx, sy, sz);
    else
        k_nodes<float><<<grid, 256, 0, c->stream>>>(
            reinterpret_cast<float*>(c->field), c->n_nodes, c->d_node_off, c->d_node_vox,
            c->d_node_sub, c->d_node_val, c->nx, c->ny, c->coef.L, nullptr, nullptr, nullptr);
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

template <typename T, int MODE_Z>
bfvm_status launch_xyz(Ctx* c, int p, const T* r, const T* cr, const T* cv)
{
    constexpr int M = MODE_Z == 0 ? 0 : 1;
    constexpr bool RN = MODE_Z == 2;
    bfvm_status st;
    if ((st = launch_nodes(c, p, RN, 0)) != BFVM_OK) return st;
    if ((st = launch_axis<T, 0, M>(c, make_args<T>(c, 0, p, r, cr, cv))) != BFVM_OK) return st;
    if ((st = launch_nodes(c, p, RN, 1)) != BFVM_OK) return st;
    if ((st = launch_axis<T, 1, M>(c, make_args<T>(c, 1, p, r, cr, cv))) != BFVM_OK) return st;
    if (c->dims == 2) return BFVM_OK;   // 2-D variant: x and y sweeps only
    if ((st = launch_nodes(c, p, RN, 2)) != BFVM_OK) return st;
    return launch_axis<T, 2, MODE_Z>(c, make_args<T>(c, 2, p, r, cr, cv));
}

}  // namespace

// The x and y sweeps of one step in the plain FP64 form, one launch per axis
// (a z-slab of a decomposed grid: its z sweep is the slabs' own, slab.cu).
bfvm_status launch_xy_plain64(Ctx* c)
{
    bfvm_status st = launch_axis<double, 0, 0>(c, make_args<double>(c, 0, 0, c->coef.r, c->coef.cr,
                                                                     c->coef.c));
    if (st != BFVM_OK) return st;
    return launch_axis<double, 1, 0>(c, make_args<double>(c, 1, 0, c->coef.r, c->coef.cr,
                                                          c->coef.c));
}

// Plain FP64 sweep along one axis from `in` to `out` (pitched layout), with
// Dirichlet mode dir_mode (see k_sweep).  Used by the adjoint.
bfvm_status launch_sweep_plain64(Ctx* c, int axis, const double* in, double* out,
                                 int dir_mode, double* out2)
{
    SweepArgs<double> A = make_args<double>(c, axis, 0, c->coef.r, c->coef.cr, c->coef.c);
    A.in = in;
    A.field = out;
    A.field2 = out2;
    c->dual_done = false;
    if (axis == 0) {
        if (dir_mode == 1) return launch_axis<double, 0, 0, 1>(c, A);
        if (dir_mode == 2) return launch_axis<double, 0, 0, 2>(c, A);
        return launch_axis<double, 0, 0, 0>(c, A);
    }
    if (axis == 1) {
        if (dir_mode == 1) return launch_axis<double, 1, 0, 1>(c, A);
        if (dir_mode == 2) return launch_axis<double, 1, 0, 2>(c, A);
        return launch_axis<double, 1, 0, 0>(c, A);
    }
    if (dir_mode == 1) return launch_axis<double, 2, 0, 1>(c, A);
    if (dir_mode == 2) return launch_axis<double, 2, 0, 2>(c, A);
    return launch_axis<double, 2, 0, 0>(c, A);
}

// Lines of each axis that need a solve in the step itself (see
// sweep_persistent.cuh): per substrate the interior of the two other
// coordinates on a Dirichlet substrate, else all of them.  Built once at
// create (the copies are synchronous, so never inside a graph capture).
bfvm_status build_line_tables(Ctx* c)
{
    if (c->n_sub > 64) return BFVM_OK;   // the generic sweep handles these
    for (int axis = 0; axis < 3; ++axis) {
        const int ea = axis == 0 ? c->ny : c->nx;   // fast other coordinate
        const int eb = axis == 2 ? c->ny : c->nz;   // slow other coordinate
        int64_t* first = c->lines_first[axis];
        first[0] = 0;
        for (int s = 0; s < c->n_sub; ++s) {
            bool dir = c->bc_kind[s] == BFVM_BC_DIRICHLET;
            // z, the slow other coordinate of the x and y lines, has boundary
            // planes only where zfaces says so: none in the 2-D variant (which
            // has no z sweep either), and only the grid's own end planes on a
            // z-slab of a decomposed grid
            const int zf = c->zfaces();
            const int b_lo = (dir && (axis == 2 || (zf & 1))) ? 1 : 0;
            const int b_hi = (dir && (axis == 2 || (zf & 2))) ? 1 : 0;
            int ca = dir ? ea - 2 : ea, cb = eb - b_lo - b_hi;
            if (ca < 0) ca = 0;
            if (cb < 0) cb = 0;
            if (c->dims == 2 && axis == 2) ca = cb = 0;
            c->lines_lo_a[axis][s] = dir ? 1 : 0;
            c->lines_cnt_a[axis][s] = ca > 0 ? ca : 1;
            c->lines_lo_b[axis][s] = b_lo;
            first[s + 1] = first[s] + (int64_t)ca * cb;
        }
        BFVM_CUDA(c, c->ensure_line_tables(axis, first));
    }
    // task list of the one-launch step: blocks of 32 lines per (axis,
    // substrate), numbered axis-major
    std::vector<int> tf(3 * c->n_sub + 1, 0);
    int64_t t = 0;
    for (int axis = 0; axis < 3; ++axis)
        for (int s = 0; s < c->n_sub; ++s) {
            tf[axis * c->n_sub + s] = (int)t;
            t += ceil_div(c->lines_first[axis][s + 1] - c->lines_first[axis][s], 32);
        }
    if (t > (int64_t)1 << 30) return BFVM_OK;   // the per-axis launches handle these
    tf[3 * c->n_sub] = (int)t;
    c->n_tasks = (int)t;
    BFVM_CUDA(c, cudaMalloc(&c->d_task_first, sizeof(int) * tf.size()));
    BFVM_CUDA(c, cudaMemcpy(c->d_task_first, tf.data(), sizeof(int) * tf.size(),
                            cudaMemcpyHostToDevice));
    const size_t nsched = 2 + 3 * (size_t)c->n_sub + 1 + (size_t)c->n_sub;
    BFVM_CUDA(c, cudaMalloc(&c->d_sched, sizeof(unsigned) * nsched));
    BFVM_CUDA(c, cudaMemset(c->d_sched, 0, sizeof(unsigned) * nsched));
    return BFVM_OK;
}

// Dirichlet nodes as the sweeps see them.
//
// A node on a face of its substrate's Dirichlet shell (one coordinate at 0 or
// n - 1 of its axis, the other two inside) is an end of the one line along
// that axis that gets a solve: the solve must take the node's value there
// instead of the boundary value (the node is applied right after the shell).
// Such values go into a per-axis end table ([line][2], NaN where the end is
// the boundary value).  Nodes on shell edges and corners lie on no solved line.
//
// For the one-launch step (sweep_step.cuh): every node goes into the
// epilogue's list, by substrate (written once all of its substrate's sweeps
// and shell are done, before its sources), and each node on a solved x or y
// line into the patch list of the sweep task of that line (written after the
// task's outputs, before its completion is published, so the next axis reads
// the node's value).  The node values before the x sweep come from one
// node-fill launch ahead of the step.
bfvm_status build_node_tables(Ctx* c, const std::vector<int64_t>& vox,
                              const std::vector<int32_t>& sub, const std::vector<double>& val,
                              const std::vector<int64_t>& off)
{
    const int64_t m = (int64_t)val.size();
    const int ext[3] = {c->nx, c->ny, c->nz};
    std::vector<double> ends[3];
    bool any_end[3] = {false, false, false};
    auto coords = [&](int64_t v, int& x, int& y, int& z) {
        x = (int)(v % c->nx);
        y = (int)((v / c->nx) % c->ny);
        z = (int)(v / ((int64_t)c->nx * c->ny));
    };
    for (int64_t i = 0; i < m; ++i) {
        const int s = sub[i];
        if (c->bc_kind[s] != BFVM_BC_DIRICHLET) continue;
        int q[3];
        coords(vox[i], q[0], q[1], q[2]);
        for (int a = 0; a < 3; ++a) {
            const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;   // the other axes
            auto inside = [&](int ax) { return q[ax] > 0 && q[ax] < ext[ax] - 1; };
            if (!inside(b1) || !inside(b2)) continue;   // no solved line along a here
            const bool lo = q[a] == 0, hi = q[a] == ext[a] - 1;
            if (!lo && !hi) continue;                   // inside the line, not an end
            if (ends[a].empty()) {
                const int64_t lines = (int64_t)c->n_sub * ext[b1] * ext[b2];
                ends[a].assign(2 * lines, (double)NAN);
            }
            int64_t fl;
            if (a == 0) fl = ((int64_t)s * c->nz + q[2]) * c->ny + q[1];
            else if (a == 1) fl = ((int64_t)s * c->nz + q[2]) * c->nx + q[0];
            else fl = ((int64_t)s * c->ny + q[1]) * c->nx + q[0];
            if (lo) ends[a][2 * fl] = val[i];
            if (hi) ends[a][2 * fl + 1] = val[i];
            any_end[a] = true;
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (!any_end[a]) continue;
        BFVM_CUDA(c, cudaMalloc(&c->d_node_ends[a], sizeof(double) * ends[a].size()));
        BFVM_CUDA(c, cudaMemcpy(c->d_node_ends[a], ends[a].data(), sizeof(double) * ends[a].size(),
                                cudaMemcpyHostToDevice));
    }
    if (c->n_tasks == 0 || !c->d_task_first) return BFVM_OK;   // no one-launch step
    // task numbering of build_line_tables
    std::vector<int64_t> tf(3 * c->n_sub + 1, 0);
    int64_t t = 0;
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < c->n_sub; ++s) {
            tf[a * c->n_sub + s] = t;
            t += ceil_div(c->lines_first[a][s + 1] - c->lines_first[a][s], 32);
        }
    std::vector<std::pair<int64_t, NodePatch>> patches;
    std::vector<std::vector<NodePatch>> by_sub(c->n_sub);
    for (int64_t i = 0; i < m; ++i) {
        const int s = sub[i];
        NodePatch np{};
        np.off = off[i];
        np.v = val[i];
        coords(vox[i], np.x, np.y, np.z);
        by_sub[s].push_back(np);
        const int q[3] = {np.x, np.y, np.z};
        for (int a = 0; a < 2; ++a) {
            // the line set of (a, s): coordinate lo_a + (t % cnt_a) of the fast
            // other axis, lo_b + (t / cnt_a) of the slow one
            const int fa = a == 0 ? q[1] : q[0];
            const int fb = q[2];
            const int lo_a = c->lines_lo_a[a][s], ca = c->lines_cnt_a[a][s];
            const int lo_b = c->lines_lo_b[a][s];
            const int64_t nl = c->lines_first[a][s + 1] - c->lines_first[a][s];
            if (fa < lo_a || fa >= lo_a + ca || fb < lo_b) continue;
            const int64_t tl = (int64_t)(fa - lo_a) + (int64_t)(fb - lo_b) * ca;
            if (tl >= nl) continue;          // on a line without a solve
            patches.push_back({tf[a * c->n_sub + s] + tl / 32, np});
        }
    }
    std::stable_sort(patches.begin(), patches.end(),
                     [](const std::pair<int64_t, NodePatch>& u,
                        const std::pair<int64_t, NodePatch>& w) { return u.first < w.first; });
    std::vector<int> first(c->n_tasks + 1, 0);
    std::vector<NodePatch> flat(patches.size());
    for (size_t i = 0; i < patches.size(); ++i) {
        first[patches[i].first + 1] += 1;
        flat[i] = patches[i].second;
    }
    for (int i = 0; i < c->n_tasks; ++i) first[i + 1] += first[i];
    std::vector<int> sfirst(c->n_sub + 1, 0);
    std::vector<NodePatch> epi;
    c->node_chunks.assign(c->n_sub, 0);
    for (int s = 0; s < c->n_sub; ++s) {
        sfirst[s] = (int)epi.size();
        epi.insert(epi.end(), by_sub[s].begin(), by_sub[s].end());
        c->node_chunks[s] = (int)ceil_div((int64_t)by_sub[s].size(), persistent::kNodeChunk);
    }
    sfirst[c->n_sub] = (int)epi.size();
    BFVM_CUDA(c, cudaMalloc(&c->d_node_task_first, sizeof(int) * first.size()));
    BFVM_CUDA(c, cudaMemcpy(c->d_node_task_first, first.data(), sizeof(int) * first.size(),
                            cudaMemcpyHostToDevice));
    BFVM_CUDA(c, cudaMalloc(&c->d_node_patch, sizeof(NodePatch) * std::max<size_t>(flat.size(), 1)));
    if (!flat.empty())
        BFVM_CUDA(c, cudaMemcpy(c->d_node_patch, flat.data(), sizeof(NodePatch) * flat.size(),
                                cudaMemcpyHostToDevice));
    BFVM_CUDA(c, cudaMalloc(&c->d_node_sfirst, sizeof(int) * sfirst.size()));
    BFVM_CUDA(c, cudaMemcpy(c->d_node_sfirst, sfirst.data(), sizeof(int) * sfirst.size(),
                            cudaMemcpyHostToDevice));
    BFVM_CUDA(c, cudaMalloc(&c->d_node_epi, sizeof(NodePatch) * std::max<size_t>(epi.size(), 1)));
    if (!epi.empty())
        BFVM_CUDA(c, cudaMemcpy(c->d_node_epi, epi.data(), sizeof(NodePatch) * epi.size(),
                                cudaMemcpyHostToDevice));
    return BFVM_OK;
}

bfvm_status launch_sources(Ctx* c, int p_next, bool renormed)
{
    const SourceTable& S = c->src;
    if (S.cap == 0) return BFVM_OK;
    // with counts only on the device, cover the capacity and let the kernel
    // read the entry count
    const int64_t* dcount = S.counts_on_host ? nullptr : S.d_count;
    const int64_t n_ent = S.counts_on_host ? S.n_entries : S.cap * c->n_sub;
    if (n_ent == 0) return BFVM_OK;
    int blk = 256;
    unsigned grid = (unsigned)ceil_div(n_ent, blk);
    int off_y = c->nx, off_z = c->nx + c->ny;
    bool scaled = (c->variant == 1 && c->precision == 64 && !renormed);
    KernelTimer timer(c, 3);
    if (c->precision == 64) {
        double* f = reinterpret_cast<double*>(c->field);
        if (scaled) {
            const double* sc = c->coef.sc + (int64_t)p_next * c->n_sub * c->coef.L;
            k_sources<double, true><<<grid, blk, 0, c->stream>>>(
                f, n_ent, dcount, S.off, S.alpha, S.beta, S.vox, S.sub, c->nx, c->ny,
                c->coef.L, off_y, off_z, sc);
        } else {
            k_sources<double, false><<<grid, blk, 0, c->stream>>>(
                f, n_ent, dcount, S.off, S.alpha, S.beta, S.vox, S.sub, c->nx, c->ny,
                c->coef.L, off_y, off_z, nullptr);
        }
    } else {
        float* f = reinterpret_cast<float*>(c->field);
        k_sources<float, false><<<grid, blk, 0, c->stream>>>(
            f, n_ent, dcount, S.off, S.alpha, S.beta, S.vox, S.sub, c->nx, c->ny,
            c->coef.L, off_y, off_z, nullptr);
    }
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

// Dirichlet shell of all Dirichlet substrates, scaled for rescale state
// p_scale (-1: plain values).
bfvm_status launch_shell_fill(Ctx* c, int p_scale)
{
    bool any = false;
    for (int s = 0; s < c->n_sub; ++s) any = any || c->bc_kind[s] == BFVM_BC_DIRICHLET;
    if (!any) return BFVM_OK;
    int64_t per = 2 * ((int64_t)c->nx * c->ny + (int64_t)c->nx * c->nz + (int64_t)c->ny * c->nz);
    int64_t n = per * c->n_sub;
    unsigned grid = (unsigned)ceil_div(n, 256);
    const double* sc = nullptr;
    if (p_scale >= 0) sc = c->coef.sc + (int64_t)p_scale * c->n_sub * c->coef.L;
    KernelTimer timer(c, 3);
    if (c->precision == 64)
        persistent::k_shell_fill<double><<<grid, 256, 0, c->stream>>>(
            reinterpret_cast<double*>(c->field), c->nx, c->ny, c->nz, c->n_sub, c->pitch,
            c->d_bc_kind, c->d_bc_value, c->coef.L, sc, c->zfaces());
    else
        persistent::k_shell_fill<float><<<grid, 256, 0, c->stream>>>(
            reinterpret_cast<float*>(c->field), c->nx, c->ny, c->nz, c->n_sub, c->pitch,
            c->d_bc_kind, c->d_bc_value, c->coef.L, nullptr, c->zfaces());
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

// One full step in rescale state p (0 <= p < period).  With renorm the z
// sweep returns the field to plain values.
bfvm_status launch_step(Ctx* c, int p, bool renorm)
{
    bfvm_status st;
    if (c->precision == 32) {
        st = launch_step_fused<float, 0>(c, 0, true, c->coef.r32, c->coef.cr32, c->coef.c32);
        if (st == BFVM_OK) return BFVM_OK;
        if (st == BFVM_ESTATE) st = launch_xyz<float, 0>(c, 0, c->coef.r32, c->coef.cr32, c->coef.c32);
        if (st != BFVM_OK) return st;
        if ((st = launch_shell_fill(c, -1)) != BFVM_OK) return st;
        if ((st = launch_nodes(c, 0, true, 3)) != BFVM_OK) return st;
        return launch_sources(c, 0, true);
    }
    if (c->variant == 0) {
        st = launch_step_fused<double, 0>(c, 0, true, c->coef.r, c->coef.cr, c->coef.c);
        if (st == BFVM_OK) return BFVM_OK;
        if (st == BFVM_ESTATE) st = launch_xyz<double, 0>(c, 0, c->coef.r, c->coef.cr, c->coef.c);
        if (st != BFVM_OK) return st;
        if ((st = launch_shell_fill(c, -1)) != BFVM_OK) return st;
        if ((st = launch_nodes(c, 0, true, 3)) != BFVM_OK) return st;
        return launch_sources(c, 0, true);
    }
    st = launch_step_fused<double, 1>(c, p, renorm, c->coef.r, c->coef.cr, c->coef.c);
    if (st == BFVM_OK) return BFVM_OK;   // sweeps, shell and sources in one launch
    if (st == BFVM_ESTATE) {
        if (renorm) st = launch_xyz<double, 2>(c, p, c->coef.r, c->coef.cr, c->coef.c);
        else st = launch_xyz<double, 1>(c, p, c->coef.r, c->coef.cr, c->coef.c);
    }
    if (st != BFVM_OK) return st;
    if ((st = launch_shell_fill(c, renorm ? -1 : p + 1)) != BFVM_OK) return st;
    if ((st = launch_nodes(c, p, renorm, 3)) != BFVM_OK) return st;
    return launch_sources(c, p + 1, renorm);
}

// ---------------------------------------------------------------- layout
namespace {

template <typename T>
__global__ void k_unscale_copy(const T* __restrict__ field, T* __restrict__ out,
                               int nx, int ny, int nz, int n_sub, int64_t pitch,
                               int64_t L, const double* __restrict__ isc)
{
    int64_t n = (int64_t)nx * ny * nz * n_sub;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    int x = (int)(e % nx);
    int64_t t = e / nx;
    int y = (int)(t % ny); t /= ny;
    int z = (int)(t % nz);
    int s = (int)(t / nz);
    int64_t src = (((int64_t)s * nz + z) * ny + y) * pitch + x;
    double val = (double)field[src];
    if (isc) {
        const double* q = isc + (int64_t)s * L;
        val = val * (q[x] * q[nx + y] * q[nx + ny + z]);
    }
    out[e] = (T)val;
}

}  // namespace

namespace {
template <typename T>
__global__ void k_check_finite(const T* __restrict__ a, int64_t n, int* flag)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite((double)a[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}
}  // namespace

// Does the dense buffer `a` (n elements of the context's type) hold a NaN or
// an Inf?  Synchronises the stream.
bfvm_status launch_check_finite(Ctx* c, const void* a, int64_t n, int* bad)
{
    BFVM_CUDA(c, cudaMemsetAsync(c->d_err + 3, 0, sizeof(int), c->stream));
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), (int64_t)c->sm_count * 8);
    if (c->precision == 64)
        k_check_finite<double><<<grid, 256, 0, c->stream>>>(static_cast<const double*>(a), n,
                                                             c->d_err + 3);
    else
        k_check_finite<float><<<grid, 256, 0, c->stream>>>(static_cast<const float*>(a), n,
                                                           c->d_err + 3);
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    BFVM_CUDA(c, cudaMemcpyAsync(bad, c->d_err + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    return BFVM_OK;
}

// Copy the field into a dense device buffer, removing the rescale of state p.
bfvm_status launch_unscale_copy(Ctx* c, void* out_dev, int p)
{
    int64_t n = (int64_t)c->nx * c->ny * c->nz * c->n_sub;
    if (n == 0) return BFVM_OK;
    const double* isc = nullptr;
    if (p != 0) isc = c->coef.isc + (int64_t)p * c->n_sub * c->coef.L;
    unsigned grid = (unsigned)ceil_div(n, 256);
    if (c->precision == 64)
        k_unscale_copy<double><<<grid, 256, 0, c->stream>>>(
            reinterpret_cast<const double*>(c->field), reinterpret_cast<double*>(out_dev),
            c->nx, c->ny, c->nz, c->n_sub, c->pitch, c->coef.L, isc);
    else
        k_unscale_copy<float><<<grid, 256, 0, c->stream>>>(
            reinterpret_cast<const float*>(c->field), reinterpret_cast<float*>(out_dev),
            c->nx, c->ny, c->nz, c->n_sub, c->pitch, c->coef.L, nullptr);
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

}  // namespace bfvm

// ================================================================ batched
// Many independent simulations of uneven sizes: one launch per phase walks a
// flat list of (member, 32-line block) tasks, one warp per task, each warp
// using the generic one-line-per-thread sweep on that member's descriptor.
namespace bfvm {
namespace {

template <typename T>
struct BatchDesc {
    SweepArgs<T> ax[3];      // state-0 arguments of the three axes
    int64_t per_state;       // n_sub * L: stride of the rescaled tables
    T* field;
    int64_t n_entries;
    const int64_t* off;
    const double* alpha;
    const double* beta;
    const int32_t* vox;
    const int32_t* sub;
    int nx, ny;
    int64_t L;
    const double* sc;        // scale tables (state 0)
    // parallel cyclic reduction of the x lines (when the batch has it):
    // per substrate (2 S + 1) x nx coefficients, stage st rows 2 st and
    // 2 st + 1 = minus the multipliers of the neighbours at -h and +h
    // (h = 2^st), row 2 S = the reciprocal of the final diagonal
    const double* pcr;       // FP64 [n_sub][2S+1][nx]
    const float* pcr32;      // FP32 [n_sub][hi, lo][2S+1][nx]
    int pcr_S;
};

template <typename T, int AXIS, int MODE>
__global__ void __launch_bounds__(256) k_batch_sweep(const BatchDesc<T>* __restrict__ D,
                                                     const int2* __restrict__ tasks,
                                                     int64_t n_tasks, int p, int max_n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (task >= n_tasks) return;
    const int2 t = tasks[task];
    SweepArgs<T> A = D[t.x].ax[AXIS];
    if (MODE >= 1) {
        const int64_t o = (int64_t)p * D[t.x].per_state;
        A.fa += o;
        A.fb += o;
        A.sc_p += o;
        A.sc_p1 += o;
        A.isc_p1 += o;
    }
    const int64_t line = (int64_t)t.y * 32 + lane;
    if (line >= A.n_lines) return;
    T* wsm = reinterpret_cast<T*>(smem_raw) + (int64_t)warp * 32 * max_n;
    sweep_one_line<T, AXIS, MODE, 0, true>(A, line, lane, wsm);
}

template <typename T, bool SCALED>
__global__ void k_batch_sources(const BatchDesc<T>* __restrict__ D,
                                const int64_t* __restrict__ prefix, int n_members,
                                int64_t total, int p_next)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    int lo = 0, hi = n_members;   // prefix[lo] <= e < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (prefix[mid] <= e) lo = mid;
        else hi = mid;
    }
    const BatchDesc<T>& d = D[lo];
    const int64_t i = e - prefix[lo];
    double b = d.beta[i];
    if (SCALED) {
        int32_t vv = d.vox[i];
        int x = vv % d.nx;
        int y = (vv / d.nx) % d.ny;
        int z = vv / (d.nx * d.ny);
        const double* q = d.sc + (int64_t)p_next * d.per_state + (int64_t)d.sub[i] * d.L;
        b *= q[x] * q[d.nx + y] * q[d.nx + d.ny + z];
    }
    T* f = d.field + d.off[i];
    *f = (T)fma(d.alpha[i], (double)*f, b);
}

// ---- parallel cyclic reduction of short x lines (batched form) ------------
// The line matrix is the same for every line of a (member, substrate), so
// the reduction's multipliers are computed once (k_pcr_coefs) and a line's
// solve is, per stage st (h = 2^st), d_k <- d_k - k1_k d_{k-h} - k2_k d_{k+h}
// (two FMAs per element), and x_k = d_k / b_k after the last stage.
struct PcrSys {
    double c, ell;   // off-diagonal magnitude and lambda dt / dims (3, or 2 in 2-D)
    int n, S;        // line length and stage count (2^S >= n)
    int64_t off;     // first double of this system in the FP64 table
};

// One CTA per system, one thread per position (n <= 128): stage by stage
// reduction of the tridiagonal matrix (diagonal 1 + ell + c at the ends,
// 1 + ell + 2c inside, off-diagonals -c) in FP64.
__global__ void k_pcr_coefs(const PcrSys* __restrict__ sys, double* __restrict__ tab,
                            float* __restrict__ tab32)
{
    __shared__ double a[128], b[128], cc[128];
    const PcrSys q = sys[blockIdx.x];
    const int n = q.n, k = threadIdx.x;
    if (k < n) {
        const int nb = (k > 0) + (k < n - 1);
        a[k] = k > 0 ? -q.c : 0.0;
        cc[k] = k < n - 1 ? -q.c : 0.0;
        b[k] = 1.0 + q.ell + q.c * (double)nb;
    }
    __syncthreads();
    double* T = tab + q.off;
    for (int st = 0; st < q.S; ++st) {
        const int h = 1 << st;
        double na = 0.0, nc = 0.0, nbv = 0.0;
        if (k < n) {
            double k1 = 0.0, k2 = 0.0;
            if (k - h >= 0) k1 = a[k] / b[k - h];
            if (k + h < n) k2 = cc[k] / b[k + h];
            na = (k - h >= 0) ? -a[k - h] * k1 : 0.0;
            nc = (k + h < n) ? -cc[k + h] * k2 : 0.0;
            nbv = b[k] - ((k - h >= 0) ? cc[k - h] * k1 : 0.0) - ((k + h < n) ? a[k + h] * k2 : 0.0);
            T[(2 * st) * n + k] = -k1;
            T[(2 * st + 1) * n + k] = -k2;
        }
        __syncthreads();
        if (k < n) {
            a[k] = na;
            cc[k] = nc;
            b[k] = nbv;
        }
        __syncthreads();
    }
    if (k < n) T[2 * q.S * n + k] = 1.0 / b[k];
    __syncthreads();
    const int rows = 2 * q.S + 1;
    float* H = tab32 + 2 * q.off;
    for (int j = k; j < rows * n; j += blockDim.x) {
        const double v = T[j];
        const float hi = (float)v;
        H[j] = hi;
        H[rows * n + j] = (float)(v - (double)hi);
    }
}

template <typename T, int E, int MODE>
__device__ __forceinline__ void pcr_stage(T (&dv)[E], const double* tb, const float* tb32,
                                          int rows_n, int n, int lane, int st)
{
    const int h = 1 << st;
    T nd[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        T dm, dp;
        if (h < 32) {
            const int sm = (lane - h) & 31, sp = (lane + h) & 31;
            const T a0 = __shfl_sync(0xffffffffu, dv[e], sm);
            const T a1 = e > 0 ? __shfl_sync(0xffffffffu, dv[e > 0 ? e - 1 : 0], sm) : (T)0;
            dm = lane >= h ? a0 : a1;
            const T b0 = __shfl_sync(0xffffffffu, dv[e], sp);
            const T b1 = e + 1 < E ? __shfl_sync(0xffffffffu, dv[e + 1 < E ? e + 1 : e], sp) : (T)0;
            dp = lane + h < 32 ? b0 : b1;
        } else {
            const int qh = h >> 5;
            dm = e >= qh ? dv[e >= qh ? e - qh : 0] : (T)0;
            dp = e + qh < E ? dv[e + qh < E ? e + qh : 0] : (T)0;
        }
        const int k = e * 32 + lane;
        nd[e] = dv[e];
        if (k < n) {
            const int j1 = (2 * st) * n + k, j2 = (2 * st + 1) * n + k;
            if (sizeof(T) == 8) {
                nd[e] = (T)fma(tb[j1], (double)dm, fma(tb[j2], (double)dp, (double)dv[e]));
            } else {
                const float t = comp_axpy(tb32[j2], tb32[rows_n + j2], (float)dp, (float)dv[e]);
                nd[e] = (T)comp_axpy(tb32[j1], tb32[rows_n + j1], (float)dm, t);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) dv[e] = nd[e];
}

// x sweep of a batch by parallel cyclic reduction: one warp per 32-line
// block task, its lines one after another, each line held as E elements
// per lane (element k in lane k mod 32, slot k / 32), so loads and stores
// are contiguous rows.  MODE 0 plain values; MODE 1 the rescaled FP64 form:
// the input is divided by this axis' scale of state p (a factor constant
// along the line passes through the solve), the output multiplied by that
// of state p + 1.  Dirichlet handling as in sweep_one_line (DIR 0).
template <typename T, int E, int MODE>
__global__ void __launch_bounds__(256) k_batch_pcr_x(const BatchDesc<T>* __restrict__ D,
                                                     const int2* __restrict__ tasks,
                                                     int64_t n_tasks, int p)
{
    const int lane = threadIdx.x & 31;
    const int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (task >= n_tasks) return;
    const int2 t = tasks[task];
    const BatchDesc<T>& d = D[t.x];
    const SweepArgs<T>& A = d.ax[0];
    const int n = A.n, S = d.pcr_S, ny = A.ny, nz = A.nz;
    const int rows_n = (2 * S + 1) * n;
    const int64_t off_p = (int64_t)p * d.per_state;
    for (int li = 0; li < 32; ++li) {
        const int64_t line = (int64_t)t.y * 32 + li;
        if (line >= A.n_lines) break;
        const int oy = (int)(line % ny);
        const int64_t tt = line / ny;
        const int oz = (int)(tt % nz);
        const int s = (int)(tt / nz);
        T* f = A.field + (((int64_t)s * nz + oz) * ny + oy) * A.pitch;
        const bool dir = A.bc_kind[s] == BFVM_BC_DIRICHLET;
        const double v = A.bc_value[s];
        const bool shell = dir && (oy == 0 || oy == ny - 1 || ((A.zfaces & 1) && oz == 0) ||
                                   ((A.zfaces & 2) && oz == nz - 1));
        const int64_t row = (int64_t)s * A.L;
        double kline = v;
        const double* scp1 = nullptr;
        const double* iscp = nullptr;
        if (MODE == 1) {
            const double* scp = A.sc_p + off_p + row;
            scp1 = A.sc_p1 + off_p + row;
            iscp = A.isc_p1 + off_p - d.per_state + row;   // inverse scales of state p
            kline = v * scp[A.off_y + oy] * scp[A.off_z + oz];
        }
        if (shell) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = e * 32 + lane;
                if (k < n) f[k] = MODE == 1 ? (T)(kline * scp1[k]) : (T)v;
            }
            continue;
        }
        T dv[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = e * 32 + lane;
            T x = (T)0;
            if (k < n) {
                x = f[k];
                if (MODE == 1) x = (T)((double)x * iscp[k]);
                if (dir && (k == 0 || k == n - 1)) x = (T)kline;
            }
            dv[e] = x;
        }
        const double* tb = d.pcr ? d.pcr + (int64_t)s * rows_n : nullptr;
        const float* tb32 = d.pcr32 ? d.pcr32 + (int64_t)s * 2 * rows_n : nullptr;
#pragma unroll
        for (int st = 0; st < 7; ++st)
            if (st < S) pcr_stage<T, E, MODE>(dv, tb, tb32, rows_n, n, lane, st);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = e * 32 + lane;
            if (k < n) {
                const int j = 2 * S * n + k;
                T x;
                if (sizeof(T) == 8) x = (T)((double)dv[e] * tb[j]);
                else x = (T)__fmaf_rn((float)dv[e], tb32[j], __fmul_rn((float)dv[e], tb32[rows_n + j]));
                if (dir && (k == 0 || k == n - 1)) x = MODE == 1 ? (T)(kline * scp1[k]) : (T)v;
                else if (MODE == 1) x = (T)((double)x * scp1[k]);
                f[k] = x;
            }
        }
    }
}

template <typename T>
bfvm_status batch_tune_t(BatchImpl* b, const std::vector<BatchDesc<T>>& desc);

// Tables of the one-launch batched step (sweep_batch_step.cuh): the groups
// (member, substrate) of the task list with their line sets, the task and
// epilogue-chunk offsets, one member table per rescale state, and the
// scheduling counters.  Leaves one_launch_ok false (the per-phase launches
// then run) where the kernel does not fit: a member without line tables,
// column buffers too long for shared memory, too many tasks.
template <typename T>
bfvm_status batch_build_one_launch(BatchImpl* b)
{
    using namespace persistent;
    constexpr int G = Groups<T>::G;
    const int M = (int)b->members.size();
    std::vector<BGroup> grp;
    std::vector<int> gmem;
    int max_n = 1;
    for (int m = 0; m < M; ++m) {
        const Ctx* c = b->members[m];
        if (c->n_sub > 64) return BFVM_OK;
        for (int a = 0; a < 3; ++a)
            if (!c->line_tables_ready[a]) return BFVM_OK;
        for (int s = 0; s < c->n_sub; ++s) gmem.push_back(m);
        max_n = std::max(max_n, std::max(c->nx, std::max(c->ny, c->nz)));
    }
    const int NS = (int)gmem.size();
    grp.resize((size_t)3 * NS);
    std::vector<int> tf((size_t)3 * NS + 1, 0);
    std::vector<int64_t> epi(NS + 1, 0);
    int64_t t = 0;
    for (int a = 0; a < 3; ++a) {
        int g = 0;
        for (int m = 0; m < M; ++m) {
            const Ctx* c = b->members[m];
            const int ext[3] = {c->nx, c->ny, c->nz};
            for (int s = 0; s < c->n_sub; ++s, ++g) {
                BGroup q;
                q.m = m;
                q.s = s;
                q.lo_a = c->lines_lo_a[a][s];
                q.cnt_a = c->lines_cnt_a[a][s];
                q.lo_b = c->lines_lo_b[a][s];
                q.n = ext[a];
                q.dir = c->bc_kind[s] == BFVM_BC_DIRICHLET ? 1 : 0;
                q.pad = 0;
                q.n_lines = c->lines_first[a][s + 1] - c->lines_first[a][s];
                q.v = c->bc_value[s];
                grp[(size_t)a * NS + g] = q;
                tf[(size_t)a * NS + g] = (int)t;
                t += ceil_div(q.n_lines, 32);
                if (t > ((int64_t)1 << 30)) return BFVM_OK;
            }
        }
    }
    tf[(size_t)3 * NS] = (int)t;
    {
        int g = 0;
        for (int m = 0; m < M; ++m) {
            const Ctx* c = b->members[m];
            const int64_t n_seg = c->src.cap > 0 ? c->src.n_seg : 0;
            for (int s = 0; s < c->n_sub; ++s, ++g)
                epi[g + 1] = epi[g] +
                             (c->bc_kind[s] == BFVM_BC_DIRICHLET
                                  ? epi_shell_chunks_z(c->nx, c->ny, c->nz, c->zfaces()) : 0) +
                             epi_src_chunks(n_seg);
        }
    }
    if (epi[NS] > ((int64_t)1 << 30)) return BFVM_OK;
    const int ns = (int)ceil_div(max_n, G) * G;
    const BatchSmem sm = batch_smem<T>(NS, ns);
    const size_t optin = b->members[0]->smem_optin;
    if (optin < sm.tab + sm.pair + 64) return BFVM_OK;
    int pairs = (int)((optin - sm.tab - 64) / sm.pair);
    if (pairs > Groups<T>::MAX_PAIRS) pairs = Groups<T>::MAX_PAIRS;
    // member tables of every rescale state of the batch
    const int P = b->period;
    std::vector<BMember<T>> mem((size_t)P * M);
    for (int p = 0; p < P; ++p) {
        const bool renorm = b->rescaled && p == P - 1;
        int g0 = 0;
        for (int m = 0; m < M; ++m) {
            Ctx* c = b->members[m];
            const T* r;
            const T* cr;
            const T* cv;
            if (sizeof(T) == 8) {
                r = reinterpret_cast<const T*>(c->coef.r);
                cr = reinterpret_cast<const T*>(c->coef.cr);
                cv = reinterpret_cast<const T*>(c->coef.c);
            } else {
                r = reinterpret_cast<const T*>(c->coef.r32);
                cr = reinterpret_cast<const T*>(c->coef.cr32);
                cv = reinterpret_cast<const T*>(c->coef.c32);
            }
            BMember<T>& d = mem[(size_t)p * M + m];
            d = BMember<T>{};
            for (int a = 0; a < 3; ++a) d.A[a] = make_args<T>(c, a, b->rescaled ? p : 0, r, cr, cv);
            EpiArgs<T>& E = d.E;
            E.field = reinterpret_cast<T*>(c->field);
            E.nx = c->nx;
            E.ny = c->ny;
            E.nz = c->nz;
            E.pitch = c->pitch;
            E.L = c->coef.L;
            E.sc = (!b->rescaled || renorm) ? nullptr : d.A[0].sc_p1;
            E.n_seg = c->src.cap > 0 ? c->src.n_seg : 0;
            E.d_nseg = nullptr;
            E.off = c->src.off;
            E.alpha = c->src.alpha;
            E.beta = c->src.beta;
            E.vox = c->src.vox;
            E.sub = c->src.sub;
            E.zf = c->zfaces();
            d.n_sub = c->n_sub;
            d.g0 = g0;
            g0 += c->n_sub;
        }
    }
    cudaError_t e;
    const size_t n_sched = 2 + (size_t)3 * NS + 1 + (size_t)NS;
    if ((e = cudaMalloc(&b->d_members, sizeof(BMember<T>) * mem.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_groups, sizeof(BGroup) * grp.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_epi_first, sizeof(int64_t) * epi.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_gmem, sizeof(int) * gmem.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_btask_first, sizeof(int) * tf.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_bsched, sizeof(unsigned) * n_sched)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess)
        return BFVM_ENOMEM;
    // synchronous copies: built once at create, outside any capture
    if ((e = cudaMemcpy(b->d_members, mem.data(), sizeof(BMember<T>) * mem.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_groups, grp.data(), sizeof(BGroup) * grp.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_epi_first, epi.data(), sizeof(int64_t) * epi.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_gmem, gmem.data(), sizeof(int) * gmem.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_btask_first, tf.data(), sizeof(int) * tf.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(b->d_bsched, 0, sizeof(unsigned) * n_sched)) != cudaSuccess ||
        (e = cudaMemset(b->d_err, 0, sizeof(int))) != cudaSuccess)
        return BFVM_ECUDA;
    b->n_groups = NS;
    b->n_btasks = (int)t;
    b->n_epi = epi[NS];
    b->b_slots = ns;
    b->b_pairs = pairs;
    b->b_smem = sm.tab + sm.pair * pairs;
    b->one_launch_ok = true;
    b->one_launch = true;
    return BFVM_OK;
}

// One step of the batch as one launch in rescale state p (sweep_batch_step.cuh).
template <typename T, int MXY, int MZ>
bfvm_status batch_step_one_launch(BatchImpl* b, int p)
{
    using namespace persistent;
    if (b->n_btasks == 0 && b->n_epi == 0) return BFVM_OK;
    const int NS = b->n_groups;
    StepSched Q;
    Q.claim = b->d_bsched;
    Q.exit_count = b->d_bsched + 1;
    Q.done = b->d_bsched + 2;
    Q.task_first = b->d_btask_first;
    Q.err = b->d_err;
    Q.n_sub = NS;
    Q.n_tasks = b->n_btasks;
    Q.max_polls = b->wait_test_polls > 0 ? (unsigned)b->wait_test_polls : kMaxPolls;
    Q.extra_need = b->wait_test_polls > 0 ? 1u : 0u;
    Q.eclaim = b->d_bsched + 2 + 3 * NS;
    Q.shell_done = Q.eclaim + 1;
    Q.n_epi_chunks = (int)b->n_epi;
    const int pairs = b->b_pairs;
    int64_t grid = ceil_div(std::max<int64_t>(b->n_btasks, 1), pairs);
    grid = std::max<int64_t>(grid, ceil_div(b->n_epi, 8 * pairs));
    const int sms = b->members[0]->sm_count;
    if (grid > sms) grid = sms;
    auto kern = k_batch_step_pair<T, MXY, MZ>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->b_smem) !=
        cudaSuccess)
        return BFVM_ECUDA;
    const size_t M = b->members.size();
    const BMember<T>* D = reinterpret_cast<const BMember<T>*>(b->d_members) + (size_t)p * M;
    kern<<<(unsigned)grid, 64 * pairs, b->b_smem, b->stream>>>(
        D, reinterpret_cast<const BGroup*>(b->d_groups), b->d_epi_first, b->d_gmem, Q, b->b_slots);
    b->launches += 1;
    return cudaGetLastError() == cudaSuccess ? BFVM_OK : BFVM_ECUDA;
}

template <typename T>
bfvm_status batch_build_t(BatchImpl* b)
{
    const int M = (int)b->members.size();
    std::vector<BatchDesc<T>> desc(M);
    std::vector<int2> tasks[3];
    std::vector<int64_t> prefix(M + 1, 0);
    int max_n = 1;
    for (int m = 0; m < M; ++m) {
        Ctx* c = b->members[m];
        const T* r;
        const T* cr;
        const T* cv;
        if (sizeof(T) == 8) {
            r = reinterpret_cast<const T*>(c->coef.r);
            cr = reinterpret_cast<const T*>(c->coef.cr);
            cv = reinterpret_cast<const T*>(c->coef.c);
        } else {
            r = reinterpret_cast<const T*>(c->coef.r32);
            cr = reinterpret_cast<const T*>(c->coef.cr32);
            cv = reinterpret_cast<const T*>(c->coef.c32);
        }
        BatchDesc<T>& d = desc[m];
        for (int a = 0; a < 3; ++a) {
            d.ax[a] = make_args<T>(c, a, 0, r, cr, cv);
            if (a >= c->dims) continue;   // a 2-D member has no z sweep
            if (d.ax[a].n > max_n) max_n = d.ax[a].n;
            int64_t nb = ceil_div(d.ax[a].n_lines, 32);
            for (int64_t k = 0; k < nb; ++k) tasks[a].push_back(make_int2(m, (int)k));
        }
        d.per_state = (int64_t)c->n_sub * c->coef.L;
        d.field = reinterpret_cast<T*>(c->field);
        d.n_entries = c->src.n_entries;
        d.off = c->src.off;
        d.alpha = c->src.alpha;
        d.beta = c->src.beta;
        d.vox = c->src.vox;
        d.sub = c->src.sub;
        d.nx = c->nx;
        d.ny = c->ny;
        d.L = c->coef.L;
        d.sc = c->coef.sc;
        prefix[m + 1] = prefix[m] + c->src.n_entries;
    }
    b->max_n = max_n;
    b->n_entries = prefix[M];
    cudaError_t e;
    // PCR stage tables of the x lines (offered when no x line is longer than
    // 128 voxels, so that a warp holds a line in at most 4 elements per lane)
    int max_nx = 0;
    for (int m = 0; m < M; ++m) max_nx = std::max(max_nx, b->members[m]->nx);
    b->pcr_ok = M > 0 && max_nx <= 128;
    if (b->pcr_ok) {
        b->pcr_e = (max_nx + 31) / 32;
        std::vector<PcrSys> sys;
        std::vector<int64_t> first(M);
        int64_t total = 0;
        for (int m = 0; m < M; ++m) {
            Ctx* c = b->members[m];
            int S = 0;
            while ((1 << S) < c->nx) ++S;
            desc[m].pcr_S = S;
            first[m] = total;
            for (int sb = 0; sb < c->n_sub; ++sb) {
                PcrSys q;
                q.c = c->D[sb] * c->dt / (c->dx * c->dx);
                q.ell = c->lambda[sb] * c->dt / (double)c->dims;   // the axis' decay share
                q.n = c->nx;
                q.S = S;
                q.off = total;
                sys.push_back(q);
                total += (int64_t)(2 * S + 1) * c->nx;
            }
        }
        PcrSys* d_sys = nullptr;
        if ((e = cudaMalloc(&b->d_pcr, sizeof(double) * total)) != cudaSuccess) return BFVM_ENOMEM;
        if ((e = cudaMalloc(&b->d_pcr32, sizeof(float) * 2 * total)) != cudaSuccess) return BFVM_ENOMEM;
        if ((e = cudaMalloc(&d_sys, sizeof(PcrSys) * sys.size())) != cudaSuccess) return BFVM_ENOMEM;
        cudaMemcpy(d_sys, sys.data(), sizeof(PcrSys) * sys.size(), cudaMemcpyHostToDevice);
        k_pcr_coefs<<<(unsigned)sys.size(), 128, 0, b->stream>>>(d_sys, b->d_pcr, b->d_pcr32);
        e = cudaStreamSynchronize(b->stream);
        cudaFree(d_sys);
        if (e != cudaSuccess) return BFVM_ECUDA;
        for (int m = 0; m < M; ++m) {
            desc[m].pcr = b->d_pcr + first[m];
            desc[m].pcr32 = b->d_pcr32 + 2 * first[m];
        }
    }
    if ((e = cudaMalloc(&b->d_desc, sizeof(BatchDesc<T>) * M)) != cudaSuccess) return BFVM_ENOMEM;
    cudaMemcpy(b->d_desc, desc.data(), sizeof(BatchDesc<T>) * M, cudaMemcpyHostToDevice);
    for (int a = 0; a < 3; ++a) {
        b->n_tasks[a] = (int64_t)tasks[a].size();
        if ((e = cudaMalloc(&b->d_tasks[a], sizeof(int2) * (tasks[a].size() + 1))) != cudaSuccess)
            return BFVM_ENOMEM;
        cudaMemcpy(b->d_tasks[a], tasks[a].data(), sizeof(int2) * tasks[a].size(),
                   cudaMemcpyHostToDevice);
    }
    if ((e = cudaMalloc(&b->d_entry_prefix, sizeof(int64_t) * (M + 1))) != cudaSuccess)
        return BFVM_ENOMEM;
    if ((e = cudaMemcpy(b->d_entry_prefix, prefix.data(), sizeof(int64_t) * (M + 1),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return BFVM_ECUDA;
    bfvm_status st = batch_tune_t<T>(b, desc);
    if (st != BFVM_OK) return st;
    return batch_build_one_launch<T>(b);
}

// Largest Thomas CTA (warps of one 32-line block each) whose line buffers
// fit in shared memory.
template <typename T>
int batch_thomas_max_warps(const BatchImpl* b)
{
    const size_t per_warp = (size_t)32 * b->max_n * sizeof(T);
    int w = (int)(b->members[0]->smem_optin / per_warp);
    return w > 8 ? 8 : w;
}

// One launch of an axis' sweep over all members with line-block shape
// (algo, warps) on the descriptors `desc` (the batch's own, or the tuner's
// copies that point at scratch fields).
template <typename T, int AXIS, int MODE>
bfvm_status batch_axis_run(BatchImpl* b, const void* desc, int p, int algo, int warps)
{
    if (b->n_tasks[AXIS] == 0) return BFVM_OK;
    const auto* D = reinterpret_cast<const BatchDesc<T>*>(desc);
    const unsigned grid = (unsigned)ceil_div(b->n_tasks[AXIS], warps);
    if (algo == 1) {
        if constexpr (AXIS == 0 && MODE <= 1) {
            if (!b->pcr_ok) return BFVM_EINVAL;
            const int2* tk = b->d_tasks[AXIS];
            const int64_t nt = b->n_tasks[AXIS];
            switch (b->pcr_e) {
                case 1: k_batch_pcr_x<T, 1, MODE><<<grid, 32 * warps, 0, b->stream>>>(D, tk, nt, p); break;
                case 2: k_batch_pcr_x<T, 2, MODE><<<grid, 32 * warps, 0, b->stream>>>(D, tk, nt, p); break;
                case 3: k_batch_pcr_x<T, 3, MODE><<<grid, 32 * warps, 0, b->stream>>>(D, tk, nt, p); break;
                default: k_batch_pcr_x<T, 4, MODE><<<grid, 32 * warps, 0, b->stream>>>(D, tk, nt, p); break;
            }
        } else {
            return BFVM_EINVAL;
        }
    } else {
        if (warps > batch_thomas_max_warps<T>(b)) return BFVM_EINVAL;
        const size_t smem = (size_t)32 * b->max_n * sizeof(T) * warps;
        auto kern = k_batch_sweep<T, AXIS, MODE>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return BFVM_ECUDA;
        kern<<<grid, 32 * warps, smem, b->stream>>>(D, b->d_tasks[AXIS], b->n_tasks[AXIS], p,
                                                     b->max_n);
    }
    return cudaGetLastError() == cudaSuccess ? BFVM_OK : BFVM_ECUDA;
}

template <typename T, int AXIS, int MODE>
bfvm_status batch_axis(BatchImpl* b, int p)
{
    if (b->n_tasks[AXIS] == 0) return BFVM_OK;
    bfvm_status st = batch_axis_run<T, AXIS, MODE>(b, b->d_desc, p, b->algo[AXIS], b->warps[AXIS]);
    if (st == BFVM_OK) b->launches += 1;
    return st;
}

// Autotuner of the line-block shapes: every candidate (Thomas with 2, 4 or
// 8 warps per CTA as far as shared memory allows; for x lines of at most
// 128 voxels also PCR with 4 or 8 warps per CTA) is launched once to warm
// up and then three times under CUDA events, on copies of the members'
// fields, in rescale state 0; the fastest shape of each axis is kept.  The
// members' own fields are not touched.  If the scratch copies cannot be
// allocated the defaults (Thomas, largest CTA) stay.
template <typename T>
bfvm_status batch_tune_t(BatchImpl* b, const std::vector<BatchDesc<T>>& desc)
{
    const int M = (int)b->members.size();
    const int wmax = batch_thomas_max_warps<T>(b);
    if (wmax < 1) return BFVM_EINVAL;
    for (int a = 0; a < 3; ++a) {
        b->algo[a] = 0;
        b->warps[a] = wmax;
        b->tune_ms[a][0] = b->tune_ms[a][1] = -1.0;
    }
    std::vector<int64_t> off(M + 1, 0);
    for (int m = 0; m < M; ++m) off[m + 1] = off[m] + b->members[m]->n_field * (int64_t)sizeof(T);
    unsigned char* scratch = nullptr;
    void* d_tune = nullptr;
    if (cudaMalloc(&scratch, off[M]) != cudaSuccess) {
        cudaGetLastError();
        return BFVM_OK;
    }
    if (cudaMalloc(&d_tune, sizeof(BatchDesc<T>) * M) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(scratch);
        return BFVM_OK;
    }
    std::vector<BatchDesc<T>> dt = desc;
    for (int m = 0; m < M; ++m) {
        T* fs = reinterpret_cast<T*>(scratch + off[m]);
        cudaMemcpyAsync(fs, b->members[m]->field, off[m + 1] - off[m], cudaMemcpyDeviceToDevice,
                        b->stream);
        for (int a = 0; a < 3; ++a) {
            dt[m].ax[a].in = fs;
            dt[m].ax[a].field = fs;
        }
        dt[m].field = fs;
    }
    cudaMemcpyAsync(d_tune, dt.data(), sizeof(BatchDesc<T>) * M, cudaMemcpyHostToDevice, b->stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto run = [&](int axis, int algo, int warps) -> bfvm_status {
        if (b->rescaled) {
            if constexpr (sizeof(T) == 8) {
                if (axis == 0) return batch_axis_run<T, 0, 1>(b, d_tune, 0, algo, warps);
                if (axis == 1) return batch_axis_run<T, 1, 1>(b, d_tune, 0, algo, warps);
                return batch_axis_run<T, 2, 1>(b, d_tune, 0, algo, warps);
            }
            return BFVM_EINVAL;
        }
        if (axis == 0) return batch_axis_run<T, 0, 0>(b, d_tune, 0, algo, warps);
        if (axis == 1) return batch_axis_run<T, 1, 0>(b, d_tune, 0, algo, warps);
        return batch_axis_run<T, 2, 0>(b, d_tune, 0, algo, warps);
    };
    for (int axis = 0; axis < 3; ++axis) {
        if (b->n_tasks[axis] == 0) continue;
        double best = 1e30;
        const int cand[5][2] = {{0, 2}, {0, 4}, {0, 8}, {1, 4}, {1, 8}};
        for (const auto& cw : cand) {
            const int algo = cw[0], warps = cw[1];
            if (algo == 0 && warps > wmax) continue;
            if (algo == 1 && (axis != 0 || !b->pcr_ok)) continue;
            if (run(axis, algo, warps) != BFVM_OK) continue;
            cudaEventRecord(e0, b->stream);
            bool ok = true;
            for (int r = 0; r < 3 && ok; ++r) ok = run(axis, algo, warps) == BFVM_OK;
            cudaEventRecord(e1, b->stream);
            if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double t = ms / 3.0;
            double& slot = b->tune_ms[axis][algo];
            if (slot < 0 || t < slot) slot = t;
            if (t < best) {
                best = t;
                b->algo[axis] = algo;
                b->warps[axis] = warps;
            }
        }
    }
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_tune);
    cudaFree(scratch);
    return cudaGetLastError() == cudaSuccess ? BFVM_OK : BFVM_ECUDA;
}

template <typename T, int MODE_Z>
bfvm_status batch_step_t(BatchImpl* b, int p)
{
    constexpr int M = MODE_Z == 0 ? 0 : 1;
    if (b->one_launch && b->one_launch_ok) return batch_step_one_launch<T, M, MODE_Z>(b, p);
    bfvm_status st;
    if ((st = batch_axis<T, 0, M>(b, p)) != BFVM_OK) return st;
    if ((st = batch_axis<T, 1, M>(b, p)) != BFVM_OK) return st;
    if ((st = batch_axis<T, 2, MODE_Z>(b, p)) != BFVM_OK) return st;
    if (b->n_entries > 0) {
        unsigned grid = (unsigned)ceil_div(b->n_entries, 256);
        const auto* D = reinterpret_cast<const BatchDesc<T>*>(b->d_desc);
        if (MODE_Z == 1)
            k_batch_sources<T, true><<<grid, 256, 0, b->stream>>>(
                D, b->d_entry_prefix, (int)b->members.size(), b->n_entries, p + 1);
        else
            k_batch_sources<T, false><<<grid, 256, 0, b->stream>>>(
                D, b->d_entry_prefix, (int)b->members.size(), b->n_entries, 0);
        b->launches += 1;
        if (cudaGetLastError() != cudaSuccess) return BFVM_ECUDA;
    }
    return BFVM_OK;
}

}  // namespace

bfvm_status batch_build(BatchImpl* b)
{
    if (b->precision == 64) return batch_build_t<double>(b);
    return batch_build_t<float>(b);
}

bfvm_status batch_launch_step(BatchImpl* b, int p, bool renorm)
{
    if (b->precision == 32) return batch_step_t<float, 0>(b, 0);
    if (!b->rescaled) return batch_step_t<double, 0>(b, 0);
    if (renorm) return batch_step_t<double, 2>(b, p);
    return batch_step_t<double, 1>(b, p);
}

bfvm_status batch_set_shape(BatchImpl* b, int axis, int algo, int warps)
{
    if (axis < 0 || axis > 2 || algo < 0 || algo > 1 || warps < 1 || warps > 8) return BFVM_EINVAL;
    if (algo == 1 && (axis != 0 || !b->pcr_ok)) return BFVM_EINVAL;
    const int wmax = b->precision == 64 ? batch_thomas_max_warps<double>(b)
                                        : batch_thomas_max_warps<float>(b);
    if (algo == 0 && warps > wmax) return BFVM_EINVAL;
    b->algo[axis] = algo;
    b->warps[axis] = warps;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_len = 0;
    return BFVM_OK;
}

void batch_free(BatchImpl* b)
{
    if (b->d_pcr) cudaFree(b->d_pcr);
    if (b->d_pcr32) cudaFree(b->d_pcr32);
    b->d_pcr = nullptr;
    b->d_pcr32 = nullptr;
    if (b->d_desc) cudaFree(b->d_desc);
    for (int a = 0; a < 3; ++a)
        if (b->d_tasks[a]) cudaFree(b->d_tasks[a]);
    if (b->d_entry_prefix) cudaFree(b->d_entry_prefix);
    void* one[] = {b->d_members, b->d_groups, b->d_epi_first, b->d_gmem, b->d_btask_first,
                   b->d_bsched, b->d_err};
    for (void* q : one)
        if (q) cudaFree(q);
    b->d_members = b->d_groups = nullptr;
    b->d_epi_first = nullptr;
    b->d_gmem = b->d_btask_first = b->d_err = nullptr;
    b->d_bsched = nullptr;
    b->one_launch_ok = b->one_launch = false;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->d_desc = nullptr;
    b->d_entry_prefix = nullptr;
    b->graph = nullptr;
}

}  // namespace bfvm
