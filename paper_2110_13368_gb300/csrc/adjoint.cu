// Reverse mode of a recorded bfvm_step(n) call.
//
// One forward step is  u1 = P(u0), v1 = A_x^{-1} u1, u2 = P(v1),
// v2 = A_y^{-1} u2, u3 = P(v2), v3 = A_z^{-1} u3, u4 = P(v3), u5 = Src(u4),
// with P the Dirichlet shell and Src the per-voxel composed cell maps.  Its
// adjoint, given g = dL/du5:
//   g <- Src^T g      (per voxel, the cells visited in reverse index order;
//                      also accumulates dL/dS_i and dL/dU_i)
//   for axis z, y, x: g <- A^{-1} (P' g) with P' zeroing the shell (the line
//                      matrices are symmetric), then
//                      dL/dlambda -= dt/3 <g, v>, dL/dD -= dt/dx^2 <g, L v>,
//                      v the raw solve output of that axis and L the
//                      zero-flux line Laplacian,
//   g <- P' g.
// Segments of k steps are replayed from their checkpoints; the replay keeps
// v1, v2, v3 (raw) and u4 of every step of the segment in device memory.
// Reductions run in FP64 with a fixed block order, so results are
// bit-reproducible run to run.
#include <math.h>

#include <vector>

#include "internal.cuh"

namespace bfvm {

namespace {

constexpr int kRedBlocks = 608;   // 4 x 152 SMs; fixed for determinism
constexpr int kRedThreads = 256;

// dense [s][z][y][x] <-> pitched copy
__global__ void k_dense_to_pitched(const double* __restrict__ src, double* __restrict__ dst,
                                   int nx, int64_t rows, int64_t pitch)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * nx) return;
    int64_t r = e / nx;
    int x = (int)(e % nx);
    dst[r * pitch + x] = src[e];
}

__global__ void k_pitched_to_dense(const double* __restrict__ src, double* __restrict__ dst,
                                   int nx, int64_t rows, int64_t pitch)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * nx) return;
    int64_t r = e / nx;
    int x = (int)(e % nx);
    dst[e] = src[r * pitch + x];
}

// out = in with the Dirichlet shell set to `value` (set = true) or zeroed
__global__ void k_shell(const double* __restrict__ in, double* __restrict__ out, int nx,
                        int ny, int nz, int n_sub, int64_t pitch,
                        const int32_t* __restrict__ kind, const double* __restrict__ value,
                        bool set)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t n = (int64_t)n_sub * nz * ny * nx;
    if (e >= n) return;
    int x = (int)(e % nx);
    int64_t t = e / nx;
    int y = (int)(t % ny); t /= ny;
    int z = (int)(t % nz);
    int s = (int)(t / nz);
    int64_t o = (((int64_t)s * nz + z) * ny + y) * pitch + x;
    double v = in[o];
    if (kind[s] == BFVM_BC_DIRICHLET &&
        (x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1))
        v = set ? value[s] : 0.0;
    out[o] = v;
}

// forward composed maps, in place: rho <- alpha rho + beta
__global__ void k_apply_maps(double* __restrict__ f, int64_t n_entries,
                             const int64_t* __restrict__ off, const double* __restrict__ alpha,
                             const double* __restrict__ beta)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_entries) return;
    f[off[e]] = fma(alpha[e], f[off[e]], beta[e]);
}

// Adjoint of the sources for one step.  Thread per (voxel segment,
// substrate): replay the cells in index order from u4 (the field before the
// sources), then walk them backwards.
__global__ void k_sources_adjoint(double* __restrict__ g, const double* __restrict__ u4,
                                  int64_t n_seg, int n_sub, const int64_t* __restrict__ seg_start,
                                  const int64_t* __restrict__ off,
                                  const int64_t* __restrict__ cell_sorted,
                                  const double* __restrict__ ca, const double* __restrict__ cb,
                                  const double* __restrict__ cw, const double* __restrict__ crs,
                                  double* __restrict__ pre, double* __restrict__ dS,
                                  double* __restrict__ dU)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_seg * n_sub) return;
    int64_t gseg = e / n_sub;
    int s = (int)(e % n_sub);
    int64_t o = off[e];
    int64_t j0 = seg_start[gseg], j1 = seg_start[gseg + 1];
    double r = u4[o];
    for (int64_t j = j0; j < j1; ++j) {
        pre[j * n_sub + s] = r;
        r = (r + ca[j * n_sub + s]) / (1.0 + cb[j * n_sub + s]);
    }
    double gr = g[o];
    for (int64_t j = j1 - 1; j >= j0; --j) {
        double b = cb[j * n_sub + s];
        double m = 1.0 / (1.0 + b);
        double fval = (pre[j * n_sub + s] + ca[j * n_sub + s]) * m;
        double ga = gr * m;
        double gb = -gr * fval * m;
        double w = cw[j];
        int64_t i = cell_sorted[j];
        dS[i * n_sub + s] += ga * w * crs[j * n_sub + s] + gb * w;
        dU[i * n_sub + s] += gb * w;
        gr = gr * m;
    }
    g[o] = gr;
}

// Per-block partial sums of <g, v> and <g, L_axis v> over substrate s.
__global__ void k_param_dots(const double* __restrict__ g, const double* __restrict__ v,
                             int axis, int s, int nx, int ny, int nz, int64_t pitch,
                             double* __restrict__ partial)
{
    __shared__ double sh0[kRedThreads];
    __shared__ double sh1[kRedThreads];
    int64_t n = (int64_t)nz * ny * nx;
    int64_t stride_a = axis == 0 ? 1 : (axis == 1 ? pitch : pitch * ny);
    int n_a = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const double* gs = g + (int64_t)s * nz * ny * pitch;
    const double* vs = v + (int64_t)s * nz * ny * pitch;
    double acc0 = 0.0, acc1 = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(e % nx);
        int64_t t = e / nx;
        int y = (int)(t % ny);
        int z = (int)(t / ny);
        int i = axis == 0 ? x : (axis == 1 ? y : z);
        int64_t o = ((int64_t)z * ny + y) * pitch + x;
        double vi = vs[o];
        double lv = 0.0;
        if (n_a > 1) {
            if (i > 0) lv += vi - vs[o - stride_a];
            if (i < n_a - 1) lv += vi - vs[o + stride_a];
        }
        double gi = gs[o];
        acc0 += gi * vi;
        acc1 += gi * lv;
    }
    sh0[threadIdx.x] = acc0;
    sh1[threadIdx.x] = acc1;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w /= 2) {
        if (threadIdx.x < w) {
            sh0[threadIdx.x] += sh0[threadIdx.x + w];
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sh0[0];
        partial[2 * blockIdx.x + 1] = sh1[0];
    }
}

// dlambda[s] -= dt/3 * sum0, dD[s] -= dt/dx^2 * sum1 (one block, fixed order)
__global__ void k_param_finish(const double* __restrict__ partial, int nblk, int s,
                               double dt, double dx, double* dD, double* dl)
{
    __shared__ double sh0[kRedThreads];
    __shared__ double sh1[kRedThreads];
    double a0 = 0.0, a1 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        a0 += partial[2 * b];
        a1 += partial[2 * b + 1];
    }
    sh0[threadIdx.x] = a0;
    sh1[threadIdx.x] = a1;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w /= 2) {
        if (threadIdx.x < w) {
            sh0[threadIdx.x] += sh0[threadIdx.x + w];
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dl[s] -= (dt / 3.0) * sh0[0];
        dD[s] -= (dt / (dx * dx)) * sh1[0];
    }
}

}  // namespace

bfvm_status run_backward(Ctx* c, const double* g_final, double* dD, double* dl,
                         double* dS, double* dU, double* g0)
{
    const int64_t rows = (int64_t)c->n_sub * c->nz * c->ny;
    const int64_t n_dense = rows * c->nx;
    const int64_t nf = c->n_field;
    const int k = c->record_every;
    const int n_steps = c->recorded_steps;
    const int n_ckpt = (int)c->checkpoints.size();
    const SourceTable& S = c->src;
    const int n_sub = c->n_sub;
    cudaStream_t st = c->stream;
    const unsigned gd = (unsigned)ceil_div(n_dense, 256);

    // device buffers
    std::vector<double*> bufs;
    auto alloc = [&](int64_t n, double** p) -> bfvm_status {
        cudaError_t e = cudaMalloc(p, sizeof(double) * (n > 0 ? n : 1));
        if (e != cudaSuccess) return cuda_err(c, e, "adjoint buffer");
        bufs.push_back(*p);
        return BFVM_OK;
    };
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (double* p : bufs) cudaFree(p);
    };
    double *g = nullptr, *cur = nullptr, *seg = nullptr, *pre = nullptr, *partial = nullptr;
    bfvm_status rc;
    if ((rc = alloc(nf, &g)) != BFVM_OK) { release(); return rc; }
    if ((rc = alloc(nf, &cur)) != BFVM_OK) { release(); return rc; }
    if ((rc = alloc(nf * 4 * (int64_t)k, &seg)) != BFVM_OK) { release(); return rc; }
    if ((rc = alloc(S.n_cells * n_sub, &pre)) != BFVM_OK) { release(); return rc; }
    if ((rc = alloc(2 * kRedBlocks, &partial)) != BFVM_OK) { release(); return rc; }
    cudaMemsetAsync(g, 0, sizeof(double) * nf, st);
    cudaMemsetAsync(cur, 0, sizeof(double) * nf, st);
    cudaMemsetAsync(dD, 0, sizeof(double) * n_sub, st);
    cudaMemsetAsync(dl, 0, sizeof(double) * n_sub, st);
    if (S.n_cells > 0) {
        cudaMemsetAsync(dS, 0, sizeof(double) * S.n_cells * n_sub, st);
        cudaMemsetAsync(dU, 0, sizeof(double) * S.n_cells * n_sub, st);
    }
    k_dense_to_pitched<<<gd, 256, 0, st>>>(g_final, g, c->nx, rows, c->pitch);
    c->launches += 1;

    auto V = [&](int t, int which) { return seg + ((int64_t)t * 4 + which) * nf; };
    for (int q = n_ckpt - 1; q >= 0; --q) {
        int t0 = q * k;
        int t1 = t0 + k < n_steps ? t0 + k : n_steps;
        k_dense_to_pitched<<<gd, 256, 0, st>>>(static_cast<const double*>(c->checkpoints[q]),
                                               cur, c->nx, rows, c->pitch);
        c->launches += 1;
        for (int t = t0; t < t1; ++t) {
            int j = t - t0;
            if ((rc = launch_sweep_plain64(c, 0, cur, V(j, 0), 1)) != BFVM_OK) break;
            if ((rc = launch_sweep_plain64(c, 1, V(j, 0), V(j, 1), 1)) != BFVM_OK) break;
            if ((rc = launch_sweep_plain64(c, 2, V(j, 1), V(j, 2), 1)) != BFVM_OK) break;
            k_shell<<<gd, 256, 0, st>>>(V(j, 2), V(j, 3), c->nx, c->ny, c->nz, n_sub, c->pitch,
                                        c->d_bc_kind, c->d_bc_value, true);
            k_shell<<<gd, 256, 0, st>>>(V(j, 2), cur, c->nx, c->ny, c->nz, n_sub, c->pitch,
                                        c->d_bc_kind, c->d_bc_value, true);
            c->launches += 2;
            if (S.n_entries > 0) {
                k_apply_maps<<<(unsigned)ceil_div(S.n_entries, 256), 256, 0, st>>>(
                    cur, S.n_entries, S.off, S.alpha, S.beta);
                c->launches += 1;
            }
        }
        if (rc != BFVM_OK) { release(); return rc; }
        for (int t = t1 - 1; t >= t0; --t) {
            int j = t - t0;
            if (S.n_entries > 0) {
                k_sources_adjoint<<<(unsigned)ceil_div(S.n_seg * n_sub, 128), 128, 0, st>>>(
                    g, V(j, 3), S.n_seg, n_sub, S.seg_start, S.off, S.cell_sorted, S.ca, S.cb,
                    S.cw, S.crs, pre, dS, dU);
                c->launches += 1;
            }
            for (int a = 2; a >= 0; --a) {
                if ((rc = launch_sweep_plain64(c, a, g, g, 2)) != BFVM_OK) break;
                for (int s = 0; s < n_sub; ++s) {
                    k_param_dots<<<kRedBlocks, kRedThreads, 0, st>>>(
                        g, V(j, a), a, s, c->nx, c->ny, c->nz, c->pitch, partial);
                    k_param_finish<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, s, c->dt,
                                                              c->dx, dD, dl);
                    c->launches += 2;
                }
            }
            if (rc != BFVM_OK) break;
            k_shell<<<gd, 256, 0, st>>>(g, g, c->nx, c->ny, c->nz, n_sub, c->pitch,
                                        c->d_bc_kind, c->d_bc_value, false);
            c->launches += 1;
        }
        if (rc != BFVM_OK) { release(); return rc; }
    }
    if (g0) {
        k_pitched_to_dense<<<gd, 256, 0, st>>>(g, g0, c->nx, rows, c->pitch);
        c->launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_err(c, e, "backward");
    return BFVM_OK;
}

}  // namespace bfvm
