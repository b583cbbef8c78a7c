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

// blocks of the parameter-dot reduction: fixed, so that the sums are the
// same bits on every run (3 x 152 SMs; on the 100^3 adjoint workload 304,
// 456, 608, 1216 and 2432 blocks gave a backward of 33.3, 32.9, 33.1, 34.3
// and 36.1 ms)
constexpr int kRedBlocks = 456;
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

// out = in with the Dirichlet shell set to `value` (set = true) or zeroed;
// out2 (may be null) receives the same values.  One thread per voxel of the
// pitched field; n_sub nz ny nx < 2^32 (32-bit index arithmetic).  dims 2:
// the shell is the four edges (the single z layer is not a boundary).
__global__ void k_shell(const double* __restrict__ in, double* __restrict__ out,
                        double* __restrict__ out2, int nx, int ny, int nz, int n_sub,
                        int64_t pitch, const int32_t* __restrict__ kind,
                        const double* __restrict__ value, bool set, int dims)
{
    const uint32_t n = (uint32_t)n_sub * nz * ny * nx;
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint32_t r = e / (uint32_t)nx;       // row (s, z, y)
    const int x = (int)(e - r * (uint32_t)nx);
    const uint32_t q = r / (uint32_t)ny;
    const int y = (int)(r - q * (uint32_t)ny);
    const uint32_t s_ = q / (uint32_t)nz;
    const int z = (int)(q - s_ * (uint32_t)nz);
    const int s = (int)s_;
    const int64_t o = (int64_t)r * pitch + x;
    double v = in[o];
    if (kind[s] == BFVM_BC_DIRICHLET &&
        (x == 0 || x == nx - 1 || y == 0 || y == ny - 1 ||
         (dims == 3 && (z == 0 || z == nz - 1))))
        v = set ? value[s] : 0.0;
    out[o] = v;
    if (out2) out2[o] = v;
}

// Dirichlet nodes on a pitched buffer f: each node entry is kept in keep
// (when not null), then set to the node's value, or to zero when val is null
// (the node projection and its adjoint).  One thread per node.
__global__ void k_node_set(double* __restrict__ f, int64_t n, const int64_t* __restrict__ off,
                           const double* __restrict__ val, double* __restrict__ keep)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = off[i];
    if (keep) keep[i] = f[o];
    f[o] = val ? val[i] : 0.0;
}

// the node entries of f back from keep
__global__ void k_node_restore(double* __restrict__ f, int64_t n,
                               const int64_t* __restrict__ off, const double* __restrict__ keep)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    f[off[i]] = keep[i];
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

// The parameter terms of one adjoint step for substrate s, all `dims` axes
// (3, or 2 for the 2-D variant: x and y) in one pass: for axis a,
// <g_a, v_a> and <g_a, L_a v_a>, with g_a the
// adjoint after the solve of axis a (gz, gy, gx) and v_a that axis' raw
// forward solve output (vx, vy, vz), L_a the zero-flux line Laplacian along
// a.  Per-block partial sums in a fixed order; the last block to finish (a
// completion counter) adds the partials in block order and applies, for
// axes z, y, x in turn, dlambda[s] -= dt/dims * <g, v> and dD[s] -= dt/dx^2
// * <g, L v>, then resets the counter.  The result is the same bits on
// every run.
__global__ void k_param_dots(const double* __restrict__ gx, const double* __restrict__ gy,
                             const double* __restrict__ gz, const double* __restrict__ vx,
                             const double* __restrict__ vy, const double* __restrict__ vz, int s,
                             int nx, int ny, int nz, int64_t pitch, double* __restrict__ partial,
                             unsigned* __restrict__ counter, double dt, double dx, double* dD,
                             double* dl, int dims)
{
    __shared__ double sh[6][kRedThreads];
    __shared__ bool last;
    const int64_t so = (int64_t)s * nz * ny * pitch;
    const int64_t stride[3] = {1, pitch, pitch * ny};
    const double* G[3] = {gx + so, gy + so, gz + so};
    const double* Vv[3] = {vx + so, vy + so, vz + so};
    double acc[6] = {0, 0, 0, 0, 0, 0};
    // Work item: 4 consecutive voxels of an x row (a quad; rows start on
    // 32-byte boundaries, the pitch being a multiple of 4).  <g, L v> is
    // summed over the edges of the line graph, (g_i - g_j)(v_i - v_j) for
    // each edge (i, j = i + 1 along the axis): the same sum as
    // sum_i g_i (L v)_i, with 4 FP64 operations per voxel and axis.
    const int nq = (nx + 3) / 4;
    const uint32_t n_quads = (uint32_t)nz * ny * nq;   // < 2^32 (32-bit index arithmetic)
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_quads;
         e += gridDim.x * blockDim.x) {
        const uint32_t r = e / (uint32_t)nq;   // row (z, y)
        const int x0 = 4 * (int)(e - r * (uint32_t)nq);
        const uint32_t zq = r / (uint32_t)ny;
        const int y = (int)(r - zq * (uint32_t)ny);
        const int z = (int)zq;
        const int64_t o = (int64_t)r * pitch + x0;
        const int cnt = min(4, nx - x0);
        const int idx[3] = {x0, y, z};
        const int ext[3] = {nx, ny, nz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a >= dims) break;
            const double* V = Vv[a] + o;
            const double* Gg = G[a] + o;
            double v[5], g[5];
            if (cnt == 4) {
                const double2 v01 = *reinterpret_cast<const double2*>(V);
                const double2 v23 = *reinterpret_cast<const double2*>(V + 2);
                const double2 g01 = *reinterpret_cast<const double2*>(Gg);
                const double2 g23 = *reinterpret_cast<const double2*>(Gg + 2);
                v[0] = v01.x; v[1] = v01.y; v[2] = v23.x; v[3] = v23.y;
                g[0] = g01.x; g[1] = g01.y; g[2] = g23.x; g[3] = g23.y;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    v[i] = i < cnt ? V[i] : 0.0;
                    g[i] = i < cnt ? Gg[i] : 0.0;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < cnt) acc[2 * a] = fma(g[i], v[i], acc[2 * a]);
            if (a == 0) {
                // edges within the quad, and to the next quad's first voxel
                const bool nxt = x0 + 4 < nx;
                v[4] = nxt ? V[4] : 0.0;
                g[4] = nxt ? Gg[4] : 0.0;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i + 1 < cnt || (i == 3 && nxt))
                        acc[1] = fma(g[i] - g[i + 1], v[i] - v[i + 1], acc[1]);
            } else if (idx[a] + 1 < ext[a]) {
                // edges to the next row (y + 1) or plane (z + 1)
                const double* V1 = V + stride[a];
                const double* G1 = Gg + stride[a];
                double v1[4], g1[4];
                if (cnt == 4) {
                    const double2 a01 = *reinterpret_cast<const double2*>(V1);
                    const double2 a23 = *reinterpret_cast<const double2*>(V1 + 2);
                    const double2 b01 = *reinterpret_cast<const double2*>(G1);
                    const double2 b23 = *reinterpret_cast<const double2*>(G1 + 2);
                    v1[0] = a01.x; v1[1] = a01.y; v1[2] = a23.x; v1[3] = a23.y;
                    g1[0] = b01.x; g1[1] = b01.y; g1[2] = b23.x; g1[3] = b23.y;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        v1[i] = i < cnt ? V1[i] : 0.0;
                        g1[i] = i < cnt ? G1[i] : 0.0;
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i < cnt) acc[2 * a + 1] = fma(g[i] - g1[i], v[i] - v1[i], acc[2 * a + 1]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w /= 2) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) partial[6 * blockIdx.x + q] = sh[q][0];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double b6[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 6; ++q) b6[q] += __ldcg(partial + 6 * b + q);
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = b6[q];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w /= 2) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int a = dims - 1; a >= 0; --a) {
            dl[s] -= (dt / (double)dims) * sh[2 * a][0];
            dD[s] -= (dt / (dx * dx)) * sh[2 * a + 1][0];
        }
        *counter = 0u;
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
    if (n_dense >= ((int64_t)1 << 32))
        return set_err(c, BFVM_EINVAL, "the adjoint covers grids of fewer than 2^32 voxel-substrates");
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
    if ((rc = alloc(6 * kRedBlocks + 1, &partial)) != BFVM_OK) { release(); return rc; }
    // the dots' completion counter lives after the partials
    unsigned* counter = reinterpret_cast<unsigned*>(partial + 6 * kRedBlocks);
    // the adjoint after the z and the y solve of a step (the x solve writes g)
    double *gz = nullptr, *gy = nullptr;
    if ((rc = alloc(nf, &gz)) != BFVM_OK) { release(); return rc; }
    if ((rc = alloc(nf, &gy)) != BFVM_OK) { release(); return rc; }
    cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    bool any_dir = false;
    for (int s = 0; s < n_sub; ++s) any_dir = any_dir || c->bc_kind[s] == BFVM_BC_DIRICHLET;
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
    // the 2-D variant sweeps x and y only; Dirichlet nodes are projected
    // like the shell (set in the replay, their adjoint zeroed)
    const int dims = c->dims;
    const int last = dims - 1;
    const int64_t nn = c->n_nodes;
    const bool nodes = nn > 0;
    const unsigned gn = (unsigned)ceil_div(nn > 0 ? nn : 1, 256);
    double* keep = nullptr;   // a buffer's node entries, kept around one solve
    if (nodes && (rc = alloc(nn, &keep)) != BFVM_OK) { release(); return rc; }
    // a projection (shell or nodes) makes the field before the sources
    // differ from the last raw solve: it is then kept apart
    const bool proj = any_dir || nodes;
    auto node_set = [&](double* f, const double* val, double* kp) {
        k_node_set<<<gn, 256, 0, c->stream>>>(f, nn, c->d_node_off, val, kp);
        c->launches += 1;
    };
    auto node_restore = [&](double* f) {
        k_node_restore<<<gn, 256, 0, c->stream>>>(f, nn, c->d_node_off, keep);
        c->launches += 1;
    };
    double* ga[3] = {g, gy, gz};   // the adjoint after the solve of each axis
    // One segment of len steps from its checkpoint (already in `cur`): the
    // replay that keeps each step's raw solve outputs and pre-source field,
    // then the adjoint steps in reverse.  Every launch reads and writes the
    // same buffers for every segment, so a segment is captured once as a
    // CUDA graph (per length) and replayed for all of them.
    auto segment = [&](int len) -> bfvm_status {
        bfvm_status r = BFVM_OK;
        for (int j = 0; j < len; ++j) {
            // the solves apply the shell to their input themselves; the
            // nodes are set in it around each solve (the raw outputs stay)
            if (nodes) node_set(cur, c->d_node_val, nullptr);
            if ((r = launch_sweep_plain64(c, 0, cur, V(j, 0), 1)) != BFVM_OK) return r;
            for (int a = 1; a <= last; ++a) {
                if (nodes) node_set(V(j, a - 1), c->d_node_val, keep);
                // without a projection the last solve also writes the next
                // step's input (cur) itself
                r = launch_sweep_plain64(c, a, V(j, a - 1), V(j, a), 1,
                                         (a == last && !proj) ? cur : nullptr);
                if (r != BFVM_OK) return r;
                if (nodes) node_restore(V(j, a - 1));
            }
            if (proj || !c->dual_done) {
                // the field before the sources: P(v_last) (kept for the
                // sources' adjoint when a projection makes it differ from
                // v_last), and the next step's input
                k_shell<<<gd, 256, 0, c->stream>>>(V(j, last), proj ? V(j, 3) : cur,
                                                   proj ? cur : nullptr, c->nx, c->ny, c->nz,
                                                   n_sub, c->pitch, c->d_bc_kind, c->d_bc_value,
                                                   true, dims);
                c->launches += 1;
                if (nodes) {
                    node_set(V(j, 3), c->d_node_val, nullptr);
                    node_set(cur, c->d_node_val, nullptr);
                }
            }
            if (S.n_entries > 0) {
                k_apply_maps<<<(unsigned)ceil_div(S.n_entries, 256), 256, 0, c->stream>>>(
                    cur, S.n_entries, S.off, S.alpha, S.beta);
                c->launches += 1;
            }
        }
        for (int j = len - 1; j >= 0; --j) {
            if (S.n_entries > 0) {
                k_sources_adjoint<<<(unsigned)ceil_div(S.n_seg * n_sub, 128), 128, 0, c->stream>>>(
                    g, proj ? V(j, 3) : V(j, last), S.n_seg, n_sub, S.seg_start, S.off,
                    S.cell_sorted, S.ca, S.cb, S.cw, S.crs, pre, dS, dU);
                c->launches += 1;
            }
            // solves of the last axis down to x, each preceded by P' (the
            // solve zeroes the shell of its input itself; the node entries
            // are zeroed around it, the dots need the unprojected adjoint)
            if (nodes) node_set(g, nullptr, nullptr);
            for (int a = last; a >= 0; --a) {
                double* in = a == last ? g : ga[a + 1];
                if (nodes && a < last) node_set(in, nullptr, keep);
                if ((r = launch_sweep_plain64(c, a, in, ga[a], 2)) != BFVM_OK) return r;
                if (nodes && a < last) node_restore(in);
            }
            for (int s = 0; s < n_sub; ++s) {
                k_param_dots<<<kRedBlocks, kRedThreads, 0, c->stream>>>(
                    g, gy, dims == 3 ? gz : gy, V(j, 0), V(j, 1), V(j, dims == 3 ? 2 : 1), s,
                    c->nx, c->ny, c->nz, c->pitch, partial, counter, c->dt, c->dx, dD, dl, dims);
                c->launches += 1;
            }
            if (any_dir) {   // P' g: the shell's adjoint is zero
                k_shell<<<gd, 256, 0, c->stream>>>(g, g, nullptr, c->nx, c->ny, c->nz, n_sub,
                                                   c->pitch, c->d_bc_kind, c->d_bc_value, false,
                                                   dims);
                c->launches += 1;
            }
            if (nodes) node_set(g, nullptr, nullptr);
        }
        return r;
    };
    // graphs of the segment lengths in use (the first segment processed,
    // the last of the run, may be shorter); launched one by one when the
    // kernels are being timed
    const bool graphs = c->use_graphs && !c->time_kernels;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int glen[2] = {0, 0};
    int64_t gkern[2] = {0, 0};   // kernels in each graph
    auto run_segment = [&](int len) -> bfvm_status {
        if (!graphs) return segment(len);
        int slot = (glen[0] == len || glen[0] == 0) ? 0 : 1;
        if (!gexec[slot]) {
            cudaStream_t cs = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamCreate");
            cudaStream_t saved = c->stream;
            const int64_t saved_launches = c->launches;
            c->stream = cs;
            bfvm_status r = BFVM_OK;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) r = cuda_err(c, e, "cudaStreamBeginCapture");
            if (r == BFVM_OK) {
                r = segment(len);
                cudaGraph_t gr = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
                if (r == BFVM_OK && e2 != cudaSuccess) r = cuda_err(c, e2, "cudaStreamEndCapture");
                if (r == BFVM_OK) {
                    e2 = cudaGraphInstantiate(&gexec[slot], gr, 0);
                    if (e2 != cudaSuccess) r = cuda_err(c, e2, "cudaGraphInstantiate");
                }
                if (gr) cudaGraphDestroy(gr);
            }
            c->stream = saved;
            cudaStreamDestroy(cs);
            gkern[slot] = c->launches - saved_launches;
            c->launches = saved_launches;
            if (r != BFVM_OK) return r;
            glen[slot] = len;
        }
        cudaError_t e = cudaGraphLaunch(gexec[slot], st);
        if (e != cudaSuccess) return cuda_err(c, e, "cudaGraphLaunch");
        c->launches += gkern[slot];
        return BFVM_OK;
    };
    for (int q = n_ckpt - 1; q >= 0; --q) {
        int t0 = q * k;
        int t1 = t0 + k < n_steps ? t0 + k : n_steps;
        k_dense_to_pitched<<<gd, 256, 0, st>>>(static_cast<const double*>(c->checkpoints[q]),
                                               cur, c->nx, rows, c->pitch);
        c->launches += 1;
        if ((rc = run_segment(t1 - t0)) != BFVM_OK) break;
    }
    cudaStreamSynchronize(st);   // before the graphs go
    for (cudaGraphExec_t ge : gexec)
        if (ge) cudaGraphExecDestroy(ge);
    if (rc != BFVM_OK) { release(); return rc; }
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
