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
constexpr uint64_t kNaIdxMask = (uint64_t(1) << bfvm::kCellIdxBits) - 1;

// keys [0, kMaxCells), flag at [kMaxCells] (as an int in the first word)
__device__ __align__(256) uint64_t g_noalloc_scratch[kMaxCells + kFlagWords];

// Device address of the scratch array, looked up once per device with that
// device current (host code sees only a host-side stand-in under the
// array's name).  The cached address belongs to the device's primary
// context: after cudaDeviceReset it is stale, so the entry point must not be
// called again in that process once the device has been reset.
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

// The first sorted position of every voxel composes that voxel's cells in
// index order into rho <- alpha rho + beta (FP64), per substrate, and
// applies it: alpha <- alpha / (1 + b_i), beta <- (beta + a_i) / (1 + b_i)
// with a_i = w S_i rho*_i, b_i = w (S_i + U_i), w = dt V_i / dx^3.
__global__ void k_na_apply(int64_t n, const uint64_t* keys, int n_sub, int64_t n_vox,
                           double dt, double vvox, const double* vol, const double* S,
                           const double* U, const double* rs, double* rho)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint64_t vox = keys[j] >> bfvm::kCellIdxBits;
    if (j > 0 && (keys[j - 1] >> bfvm::kCellIdxBits) == vox) return;
    for (int s = 0; s < n_sub; ++s) {
        double al = 1.0, be = 0.0;
        for (int64_t q = j; q < n && (keys[q] >> bfvm::kCellIdxBits) == vox; ++q) {
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
    uint64_t* keys = static_cast<uint64_t*>(base);
    int* flag = reinterpret_cast<int*>(keys + kMaxCells);

    // argument check on the device (the arrays are device memory)
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaMemsetAsync");
    bfvm::launch_validate_cells(st, n_cells, n_sub, pos, vol, S, U, rho_star, dx_um, nx, ny, nz,
                                0, nz, flag);
    int bad = 0;
    if ((e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaStreamSynchronize");
    if (bad & 1) return set_err(nullptr, BFVM_EINVAL, "cell position outside [0, n*dx] on some axis");
    if (bad & 2) return set_err(nullptr, BFVM_EINVAL, "cell volume must be finite and > 0");
    if (bad & 4) return set_err(nullptr, BFVM_EINVAL, "secretion/uptake rates must be finite and >= 0");
    if (bad & 8) return set_err(nullptr, BFVM_EINVAL, "rho_star must be finite");

    int64_t n_pad = bfvm::kCellSortBlock;
    while (n_pad < n_cells) n_pad *= 2;
    bfvm::launch_cell_keys(st, n_cells, n_pad, pos, dx_um, nx, ny, nz, 0, nz, keys);
    bfvm::launch_sort_keys(st, keys, n_pad);
    k_na_apply<<<(unsigned)bfvm::ceil_div(n_cells, 128), 128, 0, st>>>(
        n_cells, keys, n_sub, n_vox, dt_min, dx_um * dx_um * dx_um, vol, S, U, rho_star, rho);
    if ((e = cudaGetLastError()) != cudaSuccess) return bfvm::cuda_err(nullptr, e, "launch");
    return BFVM_OK;
}
