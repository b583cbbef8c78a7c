// One grid decomposed along z over several contexts (the multi-GPU
// direction of the paper's "Introduction and Motivation" and "Future Work":
// an MPI+X split of the domain), one z-slab per context, usually one context
// per GPU.
//
// The x and y lines of a slab lie inside it and are swept as in any
// context.  A z line crosses every slab; its solve is the Thomas algorithm
// of the whole line, split into the slabs' segments through the affine form
// of its two recurrences (the same algebra as the split line solve of
// sweep_split.cuh):
//   forward   d'_k = r_k d_k + m_k d'_{k-1},   m_k = c r_k,
//   backward  x_k  = d'_k + m_k x_{k+1}.
// Run from a zero incoming value over slab j, the forward gives f_k and the
// true d'_k = f_k + G_k D_j (G_k the product of the m_i from the slab's first
// layer to k, D_j the true d' just below the slab); the backward from zero
// gives g_k and the true x_k = g_k + S_k X_j (S_k the product from k to the
// slab's last layer, X_j the true x just above it).  Both D_j and X_j follow
// from the other slabs' end values by the same affine rule, with P_j the
// product of all m_i of slab j:
//   D_{j+1} = f_last(j) + P_j D_j,  D_0 = 0;   X_{j-1} = g_first(j) + P_j X_j,
//   X_{last} = 0.
// So a step on a slab runs in three calls with one exchange of one value
// per z line and substrate between them:
//   bfvm_slab_forward   the x and y sweeps (with their Dirichlet handling),
//                       then the z forward from zero; f_last to the send
//                       buffer;
//   (the caller gathers every slab's send buffer, in slab order)
//   bfvm_slab_backward  D from the gathered values, the correction, the
//                       backward from zero; g_first to the send buffer;
//   (gather again)
//   bfvm_slab_finish    X, x = g + S X, the Dirichlet ends of the grid, the
//                       Dirichlet shell of the slab and its cells' sources.
// The z coefficients are those of the whole line (the end rows of the line
// matrix belong to the first and the last slab only) and are built on the
// GPU at create, in FP64, with the slab products.
//
// A slab context is FP64 in the plain Thomas form; it cannot record for the
// adjoint, hold Dirichlet nodes, take the 2-D option or join a batch.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bfvm {
namespace {

// Slab tables, FP64, [kind][s][nz] for kind 0 r = 1/den, 1 m = c/den,
// 2 G (prefix products of m within the slab), 3 S (suffix products), then
// [s][n_slabs] the product P_j of every slab, then c per substrate.
struct SlabTab {
    const double* r;
    const double* m;
    const double* G;
    const double* S;
    const double* P;
    const double* c;
};

__host__ __device__ inline SlabTab slab_tab(const double* base, int n_sub, int nz, int n_slabs)
{
    const int64_t blk = (int64_t)n_sub * nz;
    const double* P = base + 4 * blk;
    return SlabTab{base, base + blk, base + 2 * blk, base + 3 * blk, P,
                   P + (int64_t)n_sub * n_slabs};
}

inline size_t slab_tab_doubles(int n_sub, int nz, int n_slabs)
{
    return (size_t)4 * n_sub * nz + (size_t)n_sub * n_slabs + (size_t)n_sub;
}

// One thread per substrate walks the whole z line: Thomas pivots of the
// line matrix (diagonal 1 + ell + c at the line's ends, 1 + ell + 2c inside,
// off-diagonals -c; 1 + ell for a line of one layer), and the products.
__global__ void k_slab_tables(int n_sub, int nz_global, int n_slabs, const int* z_starts,
                              int slab, double dt, double dx, const double* D,
                              const double* lambda, double* tab)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sub) return;
    const int z0 = z_starts[slab], nzl = z_starts[slab + 1] - z0;
    double* r = tab;
    double* m = tab + (int64_t)n_sub * nzl;
    double* G = m + (int64_t)n_sub * nzl;
    double* S = G + (int64_t)n_sub * nzl;
    double* P = S + (int64_t)n_sub * nzl;
    double* cv = P + (int64_t)n_sub * n_slabs;
    const double c = D[s] * dt / (dx * dx);
    const double ell = lambda[s] * dt / 3.0;
    cv[s] = c;
    double den = 1.0;
    int j = 0;
    double prod = 1.0;
    for (int k = 0; k < nz_global; ++k) {
        const int nb = (k > 0) + (k < nz_global - 1);   // neighbours along the line
        const double b = 1.0 + ell + c * (double)nb;
        den = (k == 0) ? b : b - c * (c / den);
        const double rk = 1.0 / den;
        const double mk = c / den;
        while (k >= z_starts[j + 1]) {   // k enters slab j + 1
            P[(int64_t)s * n_slabs + j] = prod;
            prod = 1.0;
            ++j;
        }
        prod *= mk;
        if (k >= z0 && k < z0 + nzl) {
            const int64_t i = (int64_t)s * nzl + (k - z0);
            r[i] = rk;
            m[i] = mk;
            G[i] = (k == z0) ? mk : G[i - 1] * mk;
        }
    }
    P[(int64_t)s * n_slabs + j] = prod;
    for (int k = nzl - 1; k >= 0; --k) {
        const int64_t i = (int64_t)s * nzl + k;
        S[i] = (k == nzl - 1) ? m[i] : m[i] * S[i + 1];
    }
}

struct SlabArgs {
    double* field;
    int nx, ny, nzl, n_sub;
    int64_t pitch;
    const int32_t* bc_kind;
    const double* bc_value;
    bool first, last;     // the slab holds the grid's z = 0 / z = nz_global - 1 layer
    int slab, n_slabs;
    SlabTab t;
    double* send;         // [n_sub][ny][nx], the caller's
    const double* recv;   // [n_slabs][n_sub][ny][nx]
};

// Column (z line) of thread i: substrate, x, y; false past the last one.
// all_shell: the column lies on the Dirichlet shell (x or y on the face):
// the shell fill writes it, no solve.
__device__ __forceinline__ bool slab_column(const SlabArgs& A, int64_t i, int& s, int& x, int& y,
                                            int64_t& base, bool& dir, bool& all_shell)
{
    const int64_t plane = (int64_t)A.nx * A.ny;
    if (i >= plane * A.n_sub) return false;
    s = (int)(i / plane);
    const int64_t q = i - (int64_t)s * plane;
    y = (int)(q / A.nx);
    x = (int)(q - (int64_t)y * A.nx);
    base = ((int64_t)s * A.nzl * A.ny + y) * A.pitch + x;
    dir = A.bc_kind[s] == BFVM_BC_DIRICHLET;
    all_shell = dir && (x == 0 || x == A.nx - 1 || y == 0 || y == A.ny - 1);
    return true;
}

// 1. forward elimination of the slab's segment from a zero incoming value
__global__ void k_slab_forward(SlabArgs A)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int s, x, y;
    int64_t base;
    bool dir, all_shell;
    if (!slab_column(A, i, s, x, y, base, dir, all_shell)) return;
    if (all_shell) {
        A.send[i] = 0.0;
        return;
    }
    const int64_t stride = (int64_t)A.ny * A.pitch;
    const int64_t row = (int64_t)s * A.nzl;
    const double c = A.t.c[s];
    const double v = A.bc_value[s];
    double* f = A.field + base;
    double prev = 0.0;
    for (int k = 0; k < A.nzl; ++k) {
        double d = f[k * stride];
        if (dir && ((A.first && k == 0) || (A.last && k == A.nzl - 1))) d = v;
        prev = fma(c, prev, d) * A.t.r[row + k];
        f[k * stride] = prev;
    }
    A.send[i] = prev;
}

// 2. incoming d' of the segment from the gathered f_last of the slabs below,
// then the back substitution from zero; g_first to the send buffer
__global__ void k_slab_backward(SlabArgs A)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int s, x, y;
    int64_t base;
    bool dir, all_shell;
    if (!slab_column(A, i, s, x, y, base, dir, all_shell)) return;
    if (all_shell) {
        A.send[i] = 0.0;
        return;
    }
    const int64_t per = (int64_t)A.n_sub * A.nx * A.ny;   // one slab's values
    const double* P = A.t.P + (int64_t)s * A.n_slabs;
    double Dv = 0.0;
    for (int j = 0; j < A.slab; ++j) Dv = fma(P[j], Dv, A.recv[(int64_t)j * per + i]);
    const int64_t stride = (int64_t)A.ny * A.pitch;
    const int64_t row = (int64_t)s * A.nzl;
    double* f = A.field + base;
    double g = 0.0;
    for (int k = A.nzl - 1; k >= 0; --k) {
        const double dp = fma(A.t.G[row + k], Dv, f[k * stride]);
        g = fma(A.t.m[row + k], g, dp);
        f[k * stride] = g;
    }
    A.send[i] = g;
}

// 3. incoming x of the segment from the gathered g_first of the slabs
// above, the solution, and the Dirichlet ends of the grid's line
__global__ void k_slab_finish(SlabArgs A)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int s, x, y;
    int64_t base;
    bool dir, all_shell;
    if (!slab_column(A, i, s, x, y, base, dir, all_shell)) return;
    if (all_shell) return;
    const int64_t per = (int64_t)A.n_sub * A.nx * A.ny;
    const double* P = A.t.P + (int64_t)s * A.n_slabs;
    double X = 0.0;
    for (int j = A.n_slabs - 1; j > A.slab; --j) X = fma(P[j], X, A.recv[(int64_t)j * per + i]);
    const int64_t stride = (int64_t)A.ny * A.pitch;
    const int64_t row = (int64_t)s * A.nzl;
    const double v = A.bc_value[s];
    double* f = A.field + base;
    for (int k = 0; k < A.nzl; ++k) {
        double xv = fma(A.t.S[row + k], X, f[k * stride]);
        if (dir && ((A.first && k == 0) || (A.last && k == A.nzl - 1))) xv = v;
        f[k * stride] = xv;
    }
}

SlabArgs slab_args(Ctx* c, const double* recv, double* send)
{
    SlabArgs A;
    A.field = reinterpret_cast<double*>(c->field);
    A.nx = c->nx;
    A.ny = c->ny;
    A.nzl = c->nz;
    A.n_sub = c->n_sub;
    A.pitch = c->pitch;
    A.bc_kind = c->d_bc_kind;
    A.bc_value = c->d_bc_value;
    A.first = c->z_face_lo;
    A.last = c->z_face_hi;
    A.slab = c->slab;
    A.n_slabs = c->n_slabs;
    A.t = slab_tab(c->slab_tab, c->n_sub, c->nz, c->n_slabs);
    A.send = send;
    A.recv = recv;
    return A;
}

bfvm_status slab_launch(Ctx* c, void (*kern)(SlabArgs), const double* recv, double* send)
{
    const int64_t n = (int64_t)c->n_sub * c->nx * c->ny;
    kern<<<(unsigned)ceil_div(n, 128), 128, 0, c->stream>>>(slab_args(c, recv, send));
    c->launches += 1;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

Ctx* slab_ctx(bfvm_ctx* h)
{
    if (!h) return nullptr;
    Ctx* c = &h->impl;
    return c->slab >= 0 ? c : nullptr;
}

}  // namespace

// x and y sweeps of one step on a slab (plain FP64 form, one launch per axis)
bfvm_status launch_xy_plain64(Ctx* c);

}  // namespace bfvm

using namespace bfvm;

extern "C" {

bfvm_status bfvm_create_slab(bfvm_ctx** out, int32_t nx, int32_t ny, int32_t n_slabs,
                             const int32_t* z_starts, int32_t slab, double dx_um,
                             double dt_min, int32_t n_sub, const double* D,
                             const double* lambda, const int32_t* bc_kind,
                             const double* bc_value, void* cuda_stream)
{
    if (!out) return set_err(nullptr, BFVM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!z_starts) return set_err(nullptr, BFVM_EINVAL, "z_starts is NULL");
    if (n_slabs < 1 || n_slabs > 4096) return set_err(nullptr, BFVM_EINVAL, "n_slabs must be 1..4096");
    if (slab < 0 || slab >= n_slabs) return set_err(nullptr, BFVM_EINVAL, "slab must be 0..n_slabs-1");
    if (z_starts[0] != 0) return set_err(nullptr, BFVM_EINVAL, "z_starts[0] must be 0");
    for (int j = 0; j < n_slabs; ++j)
        if (z_starts[j + 1] <= z_starts[j])
            return set_err(nullptr, BFVM_EINVAL, "every slab needs at least one z layer");
    const int nzl = z_starts[slab + 1] - z_starts[slab];
    bfvm_ctx* h = nullptr;
    bfvm_status st = bfvm_create(&h, nx, ny, nzl, dx_um, dt_min, n_sub, D, lambda, bc_kind,
                                 bc_value, 64, cuda_stream);
    if (st != BFVM_OK) return st;
    Ctx* c = &h->impl;
    auto fail = [&](bfvm_status s) {
        set_err(nullptr, s, c->err.empty() ? "slab set-up failed" : c->err);
        bfvm_destroy(h);
        return s;
    };
    c->slab = slab;
    c->n_slabs = n_slabs;
    c->z_origin = z_starts[slab];
    c->nz_global = z_starts[n_slabs];
    c->z_face_lo = slab == 0;
    c->z_face_hi = slab == n_slabs - 1;
    c->variant = 0;       // plain Thomas form
    c->fused_step = 0;    // the z sweep is the slabs' own
    // line sets of the x and y sweeps: the slab's inner z planes are not
    // boundary planes of the grid
    c->free_line_tables();
    if ((st = build_line_tables(c)) != BFVM_OK) return fail(st);
    cudaError_t e;
    const size_t tab = sizeof(double) * slab_tab_doubles(n_sub, nzl, n_slabs);
    if ((e = cudaMalloc(&c->slab_tab, tab)) != cudaSuccess) return fail(cuda_err(c, e, "slab tables"));
    if ((e = cudaMalloc(&c->d_z_starts, sizeof(int) * (n_slabs + 1))) != cudaSuccess)
        return fail(cuda_err(c, e, "slab partition"));
    double* dD = nullptr;
    if ((e = cudaMalloc(&dD, sizeof(double) * 2 * n_sub)) != cudaSuccess)
        return fail(cuda_err(c, e, "slab parameters"));
    e = cudaMemcpy(c->d_z_starts, z_starts, sizeof(int) * (n_slabs + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dD, D, sizeof(double) * n_sub, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dD + n_sub, lambda, sizeof(double) * n_sub, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_slab_tables<<<(unsigned)ceil_div(n_sub, 64), 64, 0, c->stream>>>(
            n_sub, c->nz_global, n_slabs, c->d_z_starts, slab, dt_min, dx_um, dD, dD + n_sub,
            c->slab_tab);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dD);
    if (e != cudaSuccess) return fail(cuda_err(c, e, "slab tables"));
    *out = h;
    return BFVM_OK;
}

bfvm_status bfvm_slab_forward(bfvm_ctx* h, double* send)
{
    NvtxRange nvtx("bfvm_slab_forward");
    Ctx* c = slab_ctx(h);
    if (!c) return h ? set_err(&h->impl, BFVM_ESTATE, "not a slab context") : BFVM_EINVAL;
    if (!send) return set_err(c, BFVM_EINVAL, "send is NULL");
    bfvm_status st = launch_xy_plain64(c);
    if (st != BFVM_OK) return st;
    return slab_launch(c, k_slab_forward, nullptr, send);
}

bfvm_status bfvm_slab_backward(bfvm_ctx* h, const double* gathered, double* send)
{
    Ctx* c = slab_ctx(h);
    if (!c) return h ? set_err(&h->impl, BFVM_ESTATE, "not a slab context") : BFVM_EINVAL;
    if (!gathered || !send) return set_err(c, BFVM_EINVAL, "gathered or send is NULL");
    return slab_launch(c, k_slab_backward, gathered, send);
}

bfvm_status bfvm_slab_finish(bfvm_ctx* h, const double* gathered)
{
    NvtxRange nvtx("bfvm_slab_finish");
    Ctx* c = slab_ctx(h);
    if (!c) return h ? set_err(&h->impl, BFVM_ESTATE, "not a slab context") : BFVM_EINVAL;
    if (!gathered) return set_err(c, BFVM_EINVAL, "gathered is NULL");
    bfvm_status st = slab_launch(c, k_slab_finish, gathered, nullptr);
    if (st != BFVM_OK) return st;
    if ((st = launch_shell_fill(c, -1)) != BFVM_OK) return st;
    if ((st = launch_sources(c, 0, true)) != BFVM_OK) return st;
    c->steps_taken += 1;
    return BFVM_OK;
}

}  // extern "C"
