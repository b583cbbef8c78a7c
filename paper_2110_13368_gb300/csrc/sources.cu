// Cell sources and sinks: binning cells to voxels, ordering them by
// (voxel, cell index), and composing each voxel's cells into one affine map.
//
// The delta term of Eq. 1 applied implicitly per cell i in index order is
//   rho_v <- (rho_v + a_i) / (1 + b_i),  a_i = w_i S_i rho*_i,
//   b_i = w_i (S_i + U_i),  w_i = dt V_i / V_vox,  V_vox = dx^3.
// Maps of one voxel do not commute, so the cells of a voxel are kept in
// ascending index: the sort key is (voxel << 31) | index, unique per cell, so
// any correct sort gives that order.  The composition of the maps in that
// order is rho <- alpha rho + beta with, cell after cell,
//   alpha <- alpha / (1 + b_i),  beta <- (beta + a_i) / (1 + b_i),
// computed once here in FP64 (the paper kept this step on the host, see
// "Future Work"; here it stays on the device).
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace bfvm {

namespace {

constexpr uint64_t kIdxBits = kCellIdxBits;
constexpr uint64_t kIdxMask = (1ull << kIdxBits) - 1;

// The grid is the z-slab [z_origin, z_origin + nz) of nz_global layers
// (0 / nz for a whole grid): positions are global, each coordinate in
// [0, n_a dx] of the whole grid, and the cell's layer must lie in the slab.
__global__ void k_validate_cells(int64_t n, int n_sub, const double* pos,
                                 const double* vol, const double* S,
                                 const double* U, const double* rs, double dx, int nx,
                                 int ny, int nz, int z_origin, int nz_global, int* flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bad = 0;
    double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    if (!(px >= 0.0 && px <= nx * dx) || !(py >= 0.0 && py <= ny * dx) ||
        !(pz >= 0.0 && pz <= nz_global * dx))
        bad |= 1;
    else {
        int64_t q = (int64_t)floor(pz / dx);
        if (q > nz_global - 1) q = nz_global - 1;
        if (q < z_origin || q >= z_origin + nz) bad |= 1;
    }
    double v = vol[i];
    if (!(v > 0.0) || !isfinite(v)) bad |= 2;
    for (int s = 0; s < n_sub; ++s) {
        double a = S[i * n_sub + s], b = U[i * n_sub + s], c = rs[i * n_sub + s];
        if (!(a >= 0.0) || !isfinite(a) || !(b >= 0.0) || !isfinite(b)) bad |= 4;
        if (!isfinite(c)) bad |= 8;
    }
    if (bad) atomicOr(flag, bad);
}

__global__ void k_keys(int64_t n, int64_t n_pad, const double* pos, double dx,
                       int nx, int ny, int nz, int z_origin, int nz_global, uint64_t* keys)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    if (i >= n) {
        keys[i] = ~0ull;
        return;
    }
    int ext[3] = {nx, ny, nz_global};
    int64_t v[3];
    for (int a = 0; a < 3; ++a) {
        double q = floor(pos[3 * i + a] / dx);
        int64_t qi = (int64_t)q;
        if (qi > ext[a] - 1) qi = ext[a] - 1;
        if (qi < 0) qi = 0;
        v[a] = qi;
    }
    // the slab's own layer (clamped: a cell outside the slab is reported by
    // the check and binned to the nearest layer meanwhile)
    v[2] -= z_origin;
    if (v[2] < 0) v[2] = 0;
    if (v[2] > nz - 1) v[2] = nz - 1;
    uint64_t vox = (uint64_t)((v[2] * ny + v[1]) * (int64_t)nx + v[0]);
    keys[i] = (vox << kIdxBits) | (uint64_t)i;
}

// Bitonic sort of a power-of-two array: global passes for large strides,
// shared-memory passes once the stride fits a block of 2048 keys.
__global__ void k_bitonic_global(uint64_t* a, int64_t n, int64_t size, int64_t stride)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n / 2) return;
    int64_t i = (t / stride) * 2 * stride + (t % stride);
    int64_t j = i + stride;
    bool up = (i & size) == 0;
    uint64_t x = a[i], y = a[j];
    if ((x > y) == up) {
        a[i] = y;
        a[j] = x;
    }
}

constexpr int kSortBlock = kCellSortBlock;

// Within each block of 2048 keys: for sizes from size_lo to size_hi, strides
// down to 1 (size_lo == size_hi: only the strides < 2048 of that size).
__global__ void k_bitonic_shared(uint64_t* a, int64_t size_lo, int64_t size_hi)
{
    __shared__ uint64_t s[kSortBlock];
    int64_t base = (int64_t)blockIdx.x * kSortBlock;
    for (int k = threadIdx.x; k < kSortBlock; k += blockDim.x) s[k] = a[base + k];
    __syncthreads();
    for (int64_t size = size_lo; size <= size_hi; size *= 2) {
        int64_t st0 = size / 2;
        if (st0 >= kSortBlock) st0 = kSortBlock / 2;
        for (int64_t stride = st0; stride >= 1; stride /= 2) {
            for (int t = threadIdx.x; t < kSortBlock / 2; t += blockDim.x) {
                int i = (int)((t / stride) * 2 * stride + (t % stride));
                int j = i + (int)stride;
                bool up = ((base + i) & size) == 0;
                uint64_t x = s[i], y = s[j];
                if ((x > y) == up) {
                    s[i] = y;
                    s[j] = x;
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < kSortBlock; k += blockDim.x) a[base + k] = s[k];
}

__global__ void k_heads(int64_t n, const uint64_t* keys, int64_t* flag)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    flag[j] = (j == 0 || (keys[j] >> kIdxBits) != (keys[j - 1] >> kIdxBits)) ? 1 : 0;
}

// exclusive scan, 1024 elements per block
constexpr int kScanBlock = 1024;
__global__ void k_scan_block(const int64_t* in, int64_t* out, int64_t* sums, int64_t n)
{
    __shared__ int64_t s[kScanBlock];
    int64_t base = (int64_t)blockIdx.x * kScanBlock;
    for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x)
        s[k] = (base + k < n) ? in[base + k] : 0;
    __syncthreads();
    // Hillis-Steele inclusive scan
    for (int d = 1; d < kScanBlock; d *= 2) {
        int64_t vals[kScanBlock / 256];
        int c = 0;
        for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x, ++c)
            vals[c] = (k >= d) ? s[k - d] : 0;
        __syncthreads();
        c = 0;
        for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x, ++c) s[k] += vals[c];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x)
        if (base + k < n) out[base + k] = (k == 0 ? 0 : s[k - 1]);
    if (threadIdx.x == 0) sums[blockIdx.x] = s[kScanBlock - 1];
}

__global__ void k_scan_add(int64_t* out, const int64_t* offs, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / kScanBlock];
}

__global__ void k_segments(int64_t n, const uint64_t* keys, const int64_t* flag,
                           const int64_t* seg_id, int64_t* seg_start, int64_t* seg_vox,
                           int64_t* cell_sorted)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    cell_sorted[j] = (int64_t)(keys[j] & kIdxMask);
    if (flag[j]) {
        int64_t g = seg_id[j];
        seg_start[g] = j;
        seg_vox[g] = (int64_t)(keys[j] >> kIdxBits);
    }
}

__global__ void k_cell_terms(int64_t n, int n_sub, double dt, double vvox,
                             const int64_t* cell_sorted, const double* vol,
                             const double* S, const double* U, const double* rs,
                             double* ca, double* cb, double* cw, double* crs)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    int64_t i = cell_sorted[j];
    double w = dt * (vol[i] / vvox);
    cw[j] = w;
    for (int s = 0; s < n_sub; ++s) {
        double Si = S[i * n_sub + s], Ui = U[i * n_sub + s], ri = rs[i * n_sub + s];
        ca[j * n_sub + s] = w * Si * ri;
        cb[j * n_sub + s] = w * (Si + Ui);
        crs[j * n_sub + s] = ri;
    }
}

__global__ void k_compose(const int64_t* count, int n_sub, int nx, int ny, int nz,
                          int64_t pitch, const int64_t* seg_start,
                          const int64_t* seg_vox, const double* ca,
                          const double* cb, int64_t* off, double* alpha,
                          double* beta, int32_t* vox, int32_t* sub,
                          int64_t* seg_of_entry)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count[1]) return;
    int64_t g = e / n_sub;
    int s = (int)(e % n_sub);
    double al = 1.0, be = 0.0;
    for (int64_t j = seg_start[g]; j < seg_start[g + 1]; ++j) {
        double m = 1.0 / (1.0 + cb[j * n_sub + s]);
        al = al * m;
        be = (be + ca[j * n_sub + s]) * m;
    }
    int64_t v = seg_vox[g];
    int x = (int)(v % nx);
    int y = (int)((v / nx) % ny);
    int z = (int)(v / ((int64_t)nx * ny));
    off[e] = (((int64_t)s * nz + z) * ny + y) * pitch + x;
    alpha[e] = al;
    beta[e] = be;
    vox[e] = (int32_t)v;
    sub[e] = s;
    seg_of_entry[e] = g;
}

// Number of occupied voxels (segments) and entries, and the end of the last
// segment, from the scanned head flags.
__global__ void k_count(int64_t n, int n_sub, const int64_t* heads, const int64_t* seg_id,
                        int64_t* seg_start, int64_t* count)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t ns = seg_id[n - 1] + heads[n - 1];
    count[0] = ns;
    count[1] = ns * n_sub;
    seg_start[ns] = n;
}

// Exclusive scan with a preallocated workspace (block sums, recursively):
// no allocation and no host read.
void scan_ws(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* ws)
{
    const int64_t nb = ceil_div(n, kScanBlock);
    int64_t* sums = ws;
    int64_t* sums_scan = ws + nb + 1;
    k_scan_block<<<(unsigned)nb, 256, 0, c->stream>>>(in, out, sums, n);
    c->launches += 1;
    if (nb > 1) {
        scan_ws(c, sums, sums_scan, nb, ws + 2 * (nb + 1));
        k_scan_add<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(out, sums_scan, n);
        c->launches += 1;
    }
}

int64_t scan_ws_size(int64_t n)
{
    int64_t total = 0;
    while (true) {
        const int64_t nb = ceil_div(n, kScanBlock);
        total += 2 * (nb + 1);
        if (nb <= 1) break;
        n = nb;
    }
    return total;
}

bfvm_status sort_keys(Ctx* c, uint64_t* keys, int64_t n_pad)
{
    c->launches += launch_sort_keys(c->stream, keys, n_pad);
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

}  // namespace

// The binning and ordering kernels above, launched on a plain stream: used
// by bin_cells below and by bfvm_apply_sources_noalloc (noalloc.cu).
void launch_validate_cells(cudaStream_t st, int64_t n, int n_sub, const double* pos,
                           const double* vol, const double* S, const double* U,
                           const double* rs, double dx, int nx, int ny, int nz,
                           int z_origin, int nz_global, int* flag)
{
    k_validate_cells<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, n_sub, pos, vol, S, U, rs,
                                                                   dx, nx, ny, nz, z_origin,
                                                                   nz_global, flag);
}

void launch_cell_keys(cudaStream_t st, int64_t n, int64_t n_pad, const double* pos, double dx,
                      int nx, int ny, int nz, int z_origin, int nz_global, uint64_t* keys)
{
    k_keys<<<(unsigned)ceil_div(n_pad, 256), 256, 0, st>>>(n, n_pad, pos, dx, nx, ny, nz,
                                                           z_origin, nz_global, keys);
}

int64_t launch_sort_keys(cudaStream_t st, uint64_t* keys, int64_t n_pad)
{
    // n_pad is a power of two >= kSortBlock
    const unsigned blocks = (unsigned)(n_pad / kSortBlock);
    int64_t launches = 1;
    k_bitonic_shared<<<blocks, 512, 0, st>>>(keys, 2, kSortBlock);
    for (int64_t size = 2 * kSortBlock; size <= n_pad; size *= 2) {
        for (int64_t stride = size / 2; stride >= kSortBlock; stride /= 2) {
            k_bitonic_global<<<(unsigned)ceil_div(n_pad / 2, 256), 256, 0, st>>>(keys, n_pad, size,
                                                                                stride);
            ++launches;
        }
        k_bitonic_shared<<<blocks, 512, 0, st>>>(keys, size, size);
        ++launches;
    }
    return launches;
}

void free_sources(Ctx* c)
{
    SourceTable& S = c->src;
    void* ptrs[] = {S.off, S.alpha, S.beta, S.vox, S.sub, S.seg_start, S.seg_vox,
                    S.cell_sorted, S.ca, S.cb, S.cw, S.crs, S.seg_of_entry,
                    S.d_count, S.keys, S.heads, S.seg_id, S.scan_ws};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    S = SourceTable();
}

namespace {

// Bin, sort and compose the S.cap cells (device arrays) into the tables.
// validate_sync: check the cells first and report EINVAL synchronously
// (bfvm_set_cells); otherwise the check ORs its findings into the sticky
// device flag d_err[2], read by the next synchronising call, and nothing
// is read back (bfvm_update_cells).  Invalid positions are binned to the
// clamped voxel either way.
bfvm_status bin_cells(Ctx* c, const double* pos, const double* vol, const double* Sr,
                      const double* Ur, const double* rs, bool validate_sync)
{
    SourceTable& S = c->src;
    const int64_t n = S.cap;
    const int n_sub = c->n_sub;
    int* flag = validate_sync ? c->d_err : c->d_err + 2;
    if (validate_sync) BFVM_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    const int nzg = c->slab >= 0 ? c->nz_global : c->nz;
    launch_validate_cells(c->stream, n, n_sub, pos, vol, Sr, Ur, rs, c->dx, c->nx, c->ny, c->nz,
                          c->z_origin, nzg, flag);
    c->launches += 1;
    if (validate_sync) {
        int f = 0;
        BFVM_CUDA(c, cudaMemcpyAsync(&f, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (f & 1)
            return set_err(c, BFVM_EINVAL, c->slab >= 0 ? "cell position outside [0, n*dx] on "
                                                          "some axis, or outside this slab"
                                                        : "cell position outside [0, n*dx] on some axis");
        if (f & 2) return set_err(c, BFVM_EINVAL, "cell volume must be finite and > 0");
        if (f & 4) return set_err(c, BFVM_EINVAL, "secretion/uptake rates must be finite and >= 0");
        if (f & 8) return set_err(c, BFVM_EINVAL, "rho_star must be finite");
    }
    launch_cell_keys(c->stream, n, S.n_pad, pos, c->dx, c->nx, c->ny, c->nz, c->z_origin, nzg,
                     S.keys);
    c->launches += 1;
    bfvm_status st = sort_keys(c, S.keys, S.n_pad);
    if (st != BFVM_OK) return st;
    k_heads<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(n, S.keys, S.heads);
    c->launches += 1;
    scan_ws(c, S.heads, S.seg_id, n, S.scan_ws);
    k_count<<<1, 32, 0, c->stream>>>(n, n_sub, S.heads, S.seg_id, S.seg_start, S.d_count);
    k_segments<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(
        n, S.keys, S.heads, S.seg_id, S.seg_start, S.seg_vox, S.cell_sorted);
    k_cell_terms<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(
        n, n_sub, c->dt, c->dx * c->dx * c->dx, S.cell_sorted, vol, Sr, Ur, rs,
        S.ca, S.cb, S.cw, S.crs);
    k_compose<<<(unsigned)ceil_div(n * n_sub, 128), 128, 0, c->stream>>>(
        S.d_count, n_sub, c->nx, c->ny, c->nz, c->pitch, S.seg_start, S.seg_vox, S.ca,
        S.cb, S.off, S.alpha, S.beta, S.vox, S.sub, S.seg_of_entry);
    c->launches += 4;
    BFVM_CUDA(c, cudaGetLastError());
    return BFVM_OK;
}

}  // namespace

// pos, vol, S, U, rho_star are device pointers here.
bfvm_status build_sources(Ctx* c, int64_t n, const double* pos, const double* vol,
                          const double* Sr, const double* Ur, const double* rs)
{
    free_sources(c);
    if (n == 0) return BFVM_OK;
    if (n > (int64_t)kIdxMask)
        return set_err(c, BFVM_EINVAL, "too many cells (limit 2^31 - 1)");
    const int n_sub = c->n_sub;
    SourceTable& S = c->src;
    S.cap = n;
    S.n_cells = n;
    S.n_pad = kSortBlock;
    while (S.n_pad < n) S.n_pad *= 2;
    const int64_t ne = n * n_sub;   // at most one entry per cell and substrate
    BFVM_CUDA(c, cudaMalloc(&S.keys, sizeof(uint64_t) * S.n_pad));
    BFVM_CUDA(c, cudaMalloc(&S.heads, sizeof(int64_t) * n));
    BFVM_CUDA(c, cudaMalloc(&S.seg_id, sizeof(int64_t) * n));
    BFVM_CUDA(c, cudaMalloc(&S.scan_ws, sizeof(int64_t) * scan_ws_size(n)));
    BFVM_CUDA(c, cudaMalloc(&S.d_count, sizeof(int64_t) * 2));
    BFVM_CUDA(c, cudaMalloc(&S.seg_start, sizeof(int64_t) * (n + 1)));
    BFVM_CUDA(c, cudaMalloc(&S.seg_vox, sizeof(int64_t) * n));
    BFVM_CUDA(c, cudaMalloc(&S.cell_sorted, sizeof(int64_t) * n));
    BFVM_CUDA(c, cudaMalloc(&S.ca, sizeof(double) * n * n_sub));
    BFVM_CUDA(c, cudaMalloc(&S.cb, sizeof(double) * n * n_sub));
    BFVM_CUDA(c, cudaMalloc(&S.crs, sizeof(double) * n * n_sub));
    BFVM_CUDA(c, cudaMalloc(&S.cw, sizeof(double) * n));
    BFVM_CUDA(c, cudaMalloc(&S.off, sizeof(int64_t) * ne));
    BFVM_CUDA(c, cudaMalloc(&S.alpha, sizeof(double) * ne));
    BFVM_CUDA(c, cudaMalloc(&S.beta, sizeof(double) * ne));
    BFVM_CUDA(c, cudaMalloc(&S.vox, sizeof(int32_t) * ne));
    BFVM_CUDA(c, cudaMalloc(&S.sub, sizeof(int32_t) * ne));
    BFVM_CUDA(c, cudaMalloc(&S.seg_of_entry, sizeof(int64_t) * ne));
    bfvm_status st = bin_cells(c, pos, vol, Sr, Ur, rs, true);
    if (st != BFVM_OK) {
        free_sources(c);
        return st;
    }
    S.counts_on_host = false;
    return sync_source_counts(c);
}

bfvm_status update_sources(Ctx* c, const double* pos, const double* vol, const double* S,
                           const double* U, const double* rho_star)
{
    if (c->src.cap == 0) return set_err(c, BFVM_ESTATE, "no cells to update (bfvm_set_cells first)");
    bfvm_status st = bin_cells(c, pos, vol, S, U, rho_star, false);
    if (st != BFVM_OK) return st;
    c->src.counts_on_host = false;
    return BFVM_OK;
}

bfvm_status sync_source_counts(Ctx* c)
{
    SourceTable& S = c->src;
    if (S.counts_on_host || S.cap == 0) return BFVM_OK;
    int64_t cnt[2] = {0, 0};
    BFVM_CUDA(c, cudaMemcpyAsync(cnt, S.d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    S.n_seg = cnt[0];
    S.n_entries = cnt[1];
    S.counts_on_host = true;
    return BFVM_OK;
}

}  // namespace bfvm
