// bfvm_apply_sources_noalloc: the cell source/uptake update (the delta term
// of Eq. 1, cells in ascending index order inside each voxel) applied to a
// caller's dense device field without allocating any memory.
//
// Who needs this: code that drives many small simulations from a host loop
// and cannot afford cudaMalloc / cudaFree in that loop (cudaFree
// synchronises the whole device, and either call can stall for
// milliseconds), code that runs under a memory manager that owns every byte
// of device memory and forbids side allocations, and code with a fixed
// memory budget decided up front.  The caller passes the field and the cell
// arrays; the only scratch, the sort keys, lives in one file-scope device
// array of fixed size that every GPU loading this library reserves until
// the process exits.
//
// The scratch holds kMaxCells sort keys plus one 256-byte slot for the
// argument-check flag.  Calls on the same device share it: calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it, so order them on one stream or synchronise between them.  Every call
// clears the flag and rewrites every key it uses, so no state carries over.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "internal.cuh"

namespace {

constexpr int64_t kMaxCells = int64_t(1) << 18;       // 262,144 cells
constexpr int64_t kFlagWords = 32;                     // 256 bytes after the keys
constexpr uint64_t kNaIdxBits = 31;
constexpr uint64_t kNaIdxMask = (uint64_t(1) << kNaIdxBits) - 1;
constexpr int kNaSortBlock = 2048;

// keys [0, kMaxCells), flag at [kMaxCells] (as an int in the first word)
__device__ __align__(256) unsigned long long g_noalloc_scratch[kMaxCells + kFlagWords];

// Device address of the scratch array, looked up once per device (host code
// sees only a host-side stand-in under the array's name).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int device, void** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

__global__ void k_na_validate(int64_t n, int n_sub, const double* pos, const double* vol,
                              const double* S, const double* U, const double* rs, double lx,
                              double ly, double lz, int* flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bad = 0;
    const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    if (!(px >= 0.0 && px <= lx) || !(py >= 0.0 && py <= ly) || !(pz >= 0.0 && pz <= lz))
        bad |= 1;
    if (!(vol[i] > 0.0) || !isfinite(vol[i])) bad |= 2;
    for (int s = 0; s < n_sub; ++s) {
        const double a = S[i * n_sub + s], b = U[i * n_sub + s];
        if (!(a >= 0.0) || !isfinite(a) || !(b >= 0.0) || !isfinite(b)) bad |= 4;
        if (!isfinite(rs[i * n_sub + s])) bad |= 8;
    }
    if (bad) atomicOr(flag, bad);
}

// key = (voxel << 31) | cell index: unique, so sorting gives voxel order with
// cell-index order inside each voxel
__global__ void k_na_keys(int64_t n, int64_t n_pad, const double* pos, double dx, int nx,
                          int ny, int nz, unsigned long long* keys)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    if (i >= n) {
        keys[i] = ~0ull;
        return;
    }
    const int ext[3] = {nx, ny, nz};
    int64_t v[3];
    for (int a = 0; a < 3; ++a) {
        int64_t q = (int64_t)floor(pos[3 * i + a] / dx);
        if (q > ext[a] - 1) q = ext[a] - 1;
        if (q < 0) q = 0;
        v[a] = q;
    }
    const uint64_t vox = (uint64_t)((v[2] * ny + v[1]) * (int64_t)nx + v[0]);
    keys[i] = (vox << kNaIdxBits) | (uint64_t)i;
}

__global__ void k_na_bitonic_global(unsigned long long* a, int64_t n, int64_t size,
                                    int64_t stride)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n / 2) return;
    const int64_t i = (t / stride) * 2 * stride + (t % stride);
    const int64_t j = i + stride;
    const bool up = (i & size) == 0;
    const unsigned long long x = a[i], y = a[j];
    if ((x > y) == up) {
        a[i] = y;
        a[j] = x;
    }
}

__global__ void k_na_bitonic_shared(unsigned long long* a, int64_t size_lo, int64_t size_hi)
{
    __shared__ unsigned long long s[kNaSortBlock];
    const int64_t base = (int64_t)blockIdx.x * kNaSortBlock;
    for (int k = threadIdx.x; k < kNaSortBlock; k += blockDim.x) s[k] = a[base + k];
    __syncthreads();
    for (int64_t size = size_lo; size <= size_hi; size *= 2) {
        int64_t st0 = size / 2;
        if (st0 >= kNaSortBlock) st0 = kNaSortBlock / 2;
        for (int64_t stride = st0; stride >= 1; stride /= 2) {
            for (int t = threadIdx.x; t < kNaSortBlock / 2; t += blockDim.x) {
                const int i = (int)((t / stride) * 2 * stride + (t % stride));
                const int j = i + (int)stride;
                const bool up = ((base + i) & size) == 0;
                const unsigned long long x = s[i], y = s[j];
                if ((x > y) == up) {
                    s[i] = y;
                    s[j] = x;
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < kNaSortBlock; k += blockDim.x) a[base + k] = s[k];
}

// The first sorted position of every voxel composes that voxel's cells in
// index order into rho <- alpha rho + beta (FP64), per substrate, and
// applies it: alpha <- alpha / (1 + b_i), beta <- (beta + a_i) / (1 + b_i)
// with a_i = w S_i rho*_i, b_i = w (S_i + U_i), w = dt V_i / dx^3.
__global__ void k_na_apply(int64_t n, const unsigned long long* keys, int n_sub, int64_t n_vox,
                           double dt, double vvox, const double* vol, const double* S,
                           const double* U, const double* rs, double* rho)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint64_t vox = keys[j] >> kNaIdxBits;
    if (j > 0 && (keys[j - 1] >> kNaIdxBits) == vox) return;
    for (int s = 0; s < n_sub; ++s) {
        double al = 1.0, be = 0.0;
        for (int64_t q = j; q < n && (keys[q] >> kNaIdxBits) == vox; ++q) {
            const int64_t i = (int64_t)(keys[q] & kNaIdxMask);
            const double w = dt * (vol[i] / vvox);
            const double Si = S[i * n_sub + s], Ui = U[i * n_sub + s];
            const double a = w * Si * rs[i * n_sub + s];
            const double b = w * (Si + Ui);
            const double m = 1.0 / (1.0 + b);
            al = al * m;
            be = (be + a) * m;
        }
        double* r = rho + (int64_t)s * n_vox + (int64_t)vox;
        *r = fma(al, *r, be);
    }
}

}  // namespace

extern "C" bfvm_status bfvm_apply_sources_noalloc(double* rho, int32_t nx, int32_t ny,
                                                  int32_t nz, int32_t n_sub, double dx_um,
                                                  double dt_min, int64_t n_cells,
                                                  const double* pos, const double* vol,
                                                  const double* S, const double* U,
                                                  const double* rho_star, void* cuda_stream)
{
    using bfvm::set_err;
    if (!rho) return set_err(nullptr, BFVM_EINVAL, "rho is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || n_sub < 1)
        return set_err(nullptr, BFVM_EINVAL, "grid edges and n_sub must be >= 1");
    if (!(dx_um > 0.0) || !isfinite(dx_um) || !(dt_min > 0.0) || !isfinite(dt_min))
        return set_err(nullptr, BFVM_EINVAL, "dx and dt must be finite and > 0");
    if (n_cells < 0) return set_err(nullptr, BFVM_EINVAL, "n_cells must be >= 0");
    if (n_cells > kMaxCells)
        return set_err(nullptr, BFVM_EINVAL,
                       "bfvm_apply_sources_noalloc takes at most 262144 cells (its fixed "
                       "scratch size); use bfvm_set_cells + bfvm_step for more");
    if (n_cells == 0) return BFVM_OK;
    if (!pos || !vol || !S || !U || !rho_star)
        return set_err(nullptr, BFVM_EINVAL, "NULL cell array");
    const int64_t n_vox = (int64_t)nx * ny * nz;
    if (n_vox > (int64_t(1) << 33)) return set_err(nullptr, BFVM_EINVAL, "grid too large");

    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return bfvm::cuda_err(nullptr, e, "cudaGetDevice");
    if (device < 0 || device >= kMaxDevices)
        return set_err(nullptr, BFVM_EINVAL, "device ordinal beyond 63");
    void* base = nullptr;
    if ((e = scratch_address(device, &base)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaGetSymbolAddress");
    unsigned long long* keys = static_cast<unsigned long long*>(base);
    int* flag = reinterpret_cast<int*>(keys + kMaxCells);

    // argument check on the device (the arrays are device memory)
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaMemsetAsync");
    k_na_validate<<<(unsigned)bfvm::ceil_div(n_cells, 256), 256, 0, st>>>(
        n_cells, n_sub, pos, vol, S, U, rho_star, nx * dx_um, ny * dx_um, nz * dx_um, flag);
    int bad = 0;
    if ((e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaStreamSynchronize");
    if (bad & 1) return set_err(nullptr, BFVM_EINVAL, "cell position outside [0, n*dx] on some axis");
    if (bad & 2) return set_err(nullptr, BFVM_EINVAL, "cell volume must be finite and > 0");
    if (bad & 4) return set_err(nullptr, BFVM_EINVAL, "secretion/uptake rates must be finite and >= 0");
    if (bad & 8) return set_err(nullptr, BFVM_EINVAL, "rho_star must be finite");

    int64_t n_pad = kNaSortBlock;
    while (n_pad < n_cells) n_pad *= 2;
    k_na_keys<<<(unsigned)bfvm::ceil_div(n_pad, 256), 256, 0, st>>>(n_cells, n_pad, pos, dx_um,
                                                                     nx, ny, nz, keys);
    const unsigned blocks = (unsigned)(n_pad / kNaSortBlock);
    k_na_bitonic_shared<<<blocks, 512, 0, st>>>(keys, 2, kNaSortBlock);
    for (int64_t size = 2 * kNaSortBlock; size <= n_pad; size *= 2) {
        for (int64_t stride = size / 2; stride >= kNaSortBlock; stride /= 2)
            k_na_bitonic_global<<<(unsigned)bfvm::ceil_div(n_pad / 2, 256), 256, 0, st>>>(
                keys, n_pad, size, stride);
        k_na_bitonic_shared<<<blocks, 512, 0, st>>>(keys, size, size);
    }
    k_na_apply<<<(unsigned)bfvm::ceil_div(n_cells, 128), 128, 0, st>>>(
        n_cells, keys, n_sub, n_vox, dt_min, dx_um * dx_um * dx_um, vol, S, U, rho_star, rho);
    if ((e = cudaGetLastError()) != cudaSuccess) return bfvm::cuda_err(nullptr, e, "launch");
    return BFVM_OK;
}
