// Internal declarations shared by the CUDA translation units of libbfvm.
// Nothing here is part of the C ABI (see include/bfvm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bfvm.h"

// NVTX ranges around the ABI's long-running calls, for timelines taken with
// a profiler (NVTX v3 is header-only and costs nothing when no tool is
// attached); compiled out where the headers are missing
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define BFVM_HAVE_NVTX 1
#endif
#endif

namespace bfvm {

struct NvtxRange {
    explicit NvtxRange(const char* name)
    {
#ifdef BFVM_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange()
    {
#ifdef BFVM_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- tables
// Per substrate s and axis a (0 = x, 1 = y, 2 = z), the line matrix of that
// axis has diagonal b_i = 1 + ell + c (ends) / 1 + ell + 2c (inside), off
// diagonals -c, c = D dt / dx^2, ell = lambda dt / 3 (a line of length 1 has
// only 1 + ell).  Thomas elimination gives pivots den_0 = b_0,
// den_i = b_i - c^2 / den_{i-1}.  Tables are laid out [s][axis offset + i],
// axis offsets 0, nx, nx + ny, row length L = nx + ny + nz.
struct CoefTables {
    double* r = nullptr;    // 1 / den_i
    double* cr = nullptr;   // c / den_i
    double* c = nullptr;    // [n_sub * 3] c per substrate and axis
    // FP32 form: each coefficient as an unevaluated sum hi + lo of two
    // floats (hi = fl32(v), lo = fl32(v - hi)), so that the rounding of the
    // coefficients adds no same-sign bias to every sweep
    float* r32 = nullptr;   // [2][s][L]: hi block then lo block
    float* cr32 = nullptr;  // [2][s][L]
    float* c32 = nullptr;   // [2][s][3]
    // rescaled-Thomas tables (FP64 only), one set per rescale state p:
    // [p][s][axis offset + i]
    double* fa = nullptr;   // forward coefficient of state p
    double* fb = nullptr;   // backward coefficient of state p
    double* sc = nullptr;   // [p + 1] axis scale vector entering state p
    double* isc = nullptr;  // 1 / sc
    int period = 0;         // number of states p
    int64_t L = 0;
    // split (partitioned) line solve of the plain form: segments of seg[a]
    // elements along axis a; within each segment the prefix products
    // sg[k] = prod_{j = k0..k} cr_j and suffix products sl[k] = prod_{j =
    // k..k1-1} cr_j ([s][L]; FP32 as hi + lo blocks like cr32), and the
    // exchange buffer of the segments' end values (2 x lines x segments
    // elements of the field type)
    int seg[3] = {0, 0, 0};
    double* sg = nullptr;
    double* sl = nullptr;
    float* sg32 = nullptr;
    float* sl32 = nullptr;
    void* split_ex = nullptr;
};

// Binned cells: every voxel that holds at least one cell, with its cells'
// affine maps composed in index order.  entry e: field element offset (in
// elements, pitch layout) and rho <- alpha rho + beta.
struct SourceTable {
    int64_t n_entries = 0;
    int64_t* off = nullptr;
    double* alpha = nullptr;
    double* beta = nullptr;
    int32_t* vox = nullptr;     // voxel (x, y, z) packed as x + nx (y + ny z)
    int32_t* sub = nullptr;     // substrate of the entry
    // for the adjoint: cells sorted by (voxel, index)
    int64_t n_cells = 0;
    int64_t n_seg = 0;          // number of occupied voxels
    int64_t* seg_start = nullptr;   // [n_seg + 1] into the sorted cell list
    int64_t* seg_vox = nullptr;     // [n_seg] voxel linear index (x fastest)
    int64_t* cell_sorted = nullptr; // [n_cells] original index, sorted order
    double* ca = nullptr;       // [n_cells][n_sub] a = w S rho*, sorted order
    double* cb = nullptr;       // [n_cells][n_sub] b = w (S + U)
    double* cw = nullptr;       // [n_cells] w = dt V / V_vox
    double* crs = nullptr;      // [n_cells][n_sub] rho*
    int64_t* seg_of_entry = nullptr;  // [n_entries] segment of each entry
    // Tables are sized for `cap` cells (at most cap occupied voxels), so a
    // cell update of the same count (bfvm_update_cells) re-bins in place,
    // on the stream, without allocating or reading anything back:
    // d_count = [n_seg, n_entries] on the device; after such an update the
    // host copies n_seg / n_entries are stale (counts_on_host false) until
    // sync_source_counts() reads them.
    int64_t cap = 0;
    int64_t* d_count = nullptr;
    bool counts_on_host = true;
    int64_t n_pad = 0;
    uint64_t* keys = nullptr;   // [n_pad] sort keys
    int64_t* heads = nullptr;   // [cap] segment head flags
    int64_t* seg_id = nullptr;  // [cap] exclusive scan of the flags
    int64_t* scan_ws = nullptr; // block sums of the scan
};

// A Dirichlet node as the one-launch step writes it (sweep_step.cuh): field
// offset, raw value and coordinates (for the rescaled form's scales)
struct NodePatch {
    int64_t off;
    double v;
    int32_t x, y, z, pad;
};

struct Ctx {
    int nx = 0, ny = 0, nz = 0, n_sub = 0, precision = 64;
    int64_t pitch = 0;            // row length in elements (>= nx, multiple of 4)
    int64_t n_field = 0;          // n_sub * nz * ny * pitch
    double dx = 0, dt = 0;
    std::vector<double> D, lambda, bc_value;
    std::vector<int32_t> bc_kind;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;

    void* field = nullptr;        // T[n_field]
    int32_t* d_bc_kind = nullptr;
    double* d_bc_value = nullptr;
    float* d_bc_value32 = nullptr;
    int* d_err = nullptr;         // device error flags
    CoefTables coef;
    SourceTable src;

    int variant = 0;              // 0 plain, 1 rescaled
    int period_override = 0;
    int fuse_sources = 0;
    int use_graphs = 1;
    int grid_limit = 0;           // cap on persistent sweep CTAs (0 = one per SM)
    int sweep_kernel = 0;         // 0 warp pairs, 1 one warp per buffer
    bool dual_done = false;       // the last plain sweep also wrote its second output
    int split = 1;                // split line solve: 0 never, 1 auto, 2 always (plain form)
    int fused_step = 1;           // one launch for x, y, z: 0 never, 1 when not fewer pairs, 2 always
    int dims = 3;                 // 2: the 2-D variant (nz == 1; x and y sweeps,
                                  // lambda dt / 2 each, four-edge Dirichlet shell)
    // z-slab of a grid decomposed along z over several contexts
    // (bfvm_create_slab, slab.cu): this context holds the global z range
    // [z_origin, z_origin + nz) of nz_global layers.  z_face_lo / z_face_hi:
    // the local z = 0 / z = nz - 1 plane is a face of the whole grid (and so
    // a Dirichlet shell plane).  An ordinary context is the one slab.
    int slab = -1;                // index of this slab; -1: an ordinary context
    int n_slabs = 1;
    int z_origin = 0, nz_global = 0;
    bool z_face_lo = true, z_face_hi = true;
    // z faces that are boundary planes: bit 0 the local z = 0 plane, bit 1
    // z = nz - 1; none in the 2-D variant (its single layer is not a face)
    int zfaces() const { return dims == 2 ? 0 : ((z_face_lo ? 1 : 0) | (z_face_hi ? 2 : 0)); }
    int* d_z_starts = nullptr;    // [n_slabs + 1] first global layer of each slab
    double* slab_tab = nullptr;   // z tables of this slab (slab.cu)
    // Dirichlet nodes inside the domain (bfvm_set_dirichlet_nodes): one per
    // (voxel, substrate), the caller's later node kept where two coincide
    void* staging = nullptr;         // device buffer for unscaled copies to the host
    size_t staging_bytes = 0;
    int64_t n_nodes = 0;
    int64_t* d_node_off = nullptr;   // pitched field offset
    int32_t* d_node_vox = nullptr;   // x + nx (y + ny z)
    int32_t* d_node_sub = nullptr;
    double* d_node_val = nullptr;
    // nodes on a Dirichlet shell face: per axis, the raw values at the ends of
    // the lines they end ([line][2], NaN elsewhere; null when there are none)
    double* d_node_ends[3] = {nullptr, nullptr, nullptr};
    // the one-launch step with nodes: the patches of the x and y tasks
    // ([n_tasks + 1] first patch of each task) and every node by substrate
    // ([n_sub + 1] first node of each substrate) for the epilogue
    int* d_node_task_first = nullptr;
    NodePatch* d_node_patch = nullptr;
    int* d_node_sfirst = nullptr;
    NodePatch* d_node_epi = nullptr;
    std::vector<int> node_chunks;     // epilogue node chunks per substrate
    void free_nodes()
    {
        if (d_node_off) cudaFree(d_node_off);
        if (d_node_vox) cudaFree(d_node_vox);
        if (d_node_sub) cudaFree(d_node_sub);
        if (d_node_val) cudaFree(d_node_val);
        for (int a = 0; a < 3; ++a) {
            if (d_node_ends[a]) cudaFree(d_node_ends[a]);
            d_node_ends[a] = nullptr;
        }
        if (d_node_task_first) cudaFree(d_node_task_first);
        if (d_node_patch) cudaFree(d_node_patch);
        if (d_node_sfirst) cudaFree(d_node_sfirst);
        if (d_node_epi) cudaFree(d_node_epi);
        d_node_task_first = nullptr;
        d_node_patch = nullptr;
        d_node_sfirst = nullptr;
        d_node_epi = nullptr;
        node_chunks.clear();
        d_node_off = nullptr;
        d_node_vox = d_node_sub = nullptr;
        d_node_val = nullptr;
        n_nodes = 0;
    }
    int wait_test_polls = 0;      // > 0: the step's dependency waits cannot end and
                                  // give up after this many polls (tests only)
    int scale_state = 0;          // rescale state p of the stored field

    cudaGraphExec_t period_graph = nullptr;
    int period_graph_len = 0;
    int64_t period_graph_launches = 0;   // kernel launches captured in it

    // recording for the adjoint
    int record_every = 0;
    std::vector<void*> checkpoints;
    int recorded_steps = 0;
    bool recorded = false;

    int64_t steps_taken = 0;
    int64_t launches = 0;
    std::string err;

    // line sets of the persistent sweeps (per axis, per substrate)
    int lines_lo_a[3][64] = {}, lines_cnt_a[3][64] = {}, lines_lo_b[3][64] = {};
    int64_t lines_first[3][65] = {};
    int64_t* d_first[3] = {nullptr, nullptr, nullptr};
    int* d_lo_a[3] = {nullptr, nullptr, nullptr};
    int* d_cnt_a[3] = {nullptr, nullptr, nullptr};
    int* d_lo_b[3] = {nullptr, nullptr, nullptr};
    bool line_tables_ready[3] = {false, false, false};
    cudaError_t ensure_line_tables(int axis, const int64_t* first)
    {
        if (line_tables_ready[axis]) return cudaSuccess;
        cudaError_t e;
        if ((e = cudaMalloc(&d_first[axis], sizeof(int64_t) * (n_sub + 1))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&d_lo_a[axis], sizeof(int) * n_sub)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&d_cnt_a[axis], sizeof(int) * n_sub)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&d_lo_b[axis], sizeof(int) * n_sub)) != cudaSuccess) return e;
        // synchronous copies: the tables are built once, outside any capture
        if ((e = cudaMemcpy(d_first[axis], first, sizeof(int64_t) * (n_sub + 1),
                            cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(d_lo_a[axis], lines_lo_a[axis], sizeof(int) * n_sub,
                            cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(d_cnt_a[axis], lines_cnt_a[axis], sizeof(int) * n_sub,
                            cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(d_lo_b[axis], lines_lo_b[axis], sizeof(int) * n_sub,
                            cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        line_tables_ready[axis] = true;
        return cudaSuccess;
    }
    // task list of the one-launch step (see sweep_step.cuh): first task of
    // each (axis, substrate), and the scheduling counters [claim, exit,
    // done[3][n_sub]] (zero between launches)
    int* d_task_first = nullptr;
    unsigned* d_sched = nullptr;
    int n_tasks = 0;
    void free_line_tables()
    {
        if (d_task_first) cudaFree(d_task_first);
        if (d_sched) cudaFree(d_sched);
        d_task_first = nullptr;
        d_sched = nullptr;
        n_tasks = 0;
        for (int a = 0; a < 3; ++a) {
            if (d_first[a]) cudaFree(d_first[a]);
            if (d_lo_a[a]) cudaFree(d_lo_a[a]);
            if (d_cnt_a[a]) cudaFree(d_cnt_a[a]);
            if (d_lo_b[a]) cudaFree(d_lo_b[a]);
            d_first[a] = nullptr; d_lo_a[a] = d_cnt_a[a] = d_lo_b[a] = nullptr;
            line_tables_ready[a] = false;
        }
    }

    // optional per-kernel CUDA-event timing (kinds: 0 x, 1 y, 2 z sweep,
    // 3 sources and shell, 4 the x, y and z sweeps as one launch)
    int time_kernels = 0;
    std::vector<cudaEvent_t> ev_start, ev_stop;
    std::vector<int> ev_kind;
    double kt_ms[5] = {0, 0, 0, 0, 0};
    int64_t kt_n[5] = {0, 0, 0, 0, 0};
};

// Brackets one kernel launch with CUDA events when timing is enabled.
struct KernelTimer {
    Ctx* c;
    int kind;
    cudaEvent_t stop = nullptr;
    KernelTimer(Ctx* ctx, int k) : c(ctx), kind(k)
    {
        if (!c->time_kernels) return;
        cudaEvent_t a;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventCreate(&stop) != cudaSuccess) { cudaEventDestroy(a); stop = nullptr; return; }
        cudaEventRecord(a, c->stream);
        c->ev_start.push_back(a);
    }
    ~KernelTimer()
    {
        if (!stop) return;
        cudaEventRecord(stop, c->stream);
        c->ev_stop.push_back(stop);
        c->ev_kind.push_back(kind);
    }
};

// ------------------------------------------------------------ helpers
bfvm_status set_err(Ctx* c, bfvm_status st, const std::string& msg);
bfvm_status cuda_err(Ctx* c, cudaError_t e, const char* what);
bfvm_status check_wait_flag(Ctx* c);

#define BFVM_CUDA(ctx, call)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call); \
    } while (0)

// coefficient tables (coeffs.cu)
bfvm_status build_coefficients(Ctx* c);
void free_coefficients(Ctx* c);

// sweeps (sweeps.cu): one full step in the plain or rescaled form
bfvm_status launch_step(Ctx* c, int p, bool renorm);
bfvm_status launch_shell_fill(Ctx* c, int p_scale);
bfvm_status build_line_tables(Ctx* c);
bfvm_status launch_unscale_copy(Ctx* c, void* out_dev, int p);
bfvm_status launch_check_finite(Ctx* c, const void* a, int64_t n, int* bad);

// sources (sources.cu)
bfvm_status build_sources(Ctx* c, int64_t n_cells, const double* pos,
                          const double* vol, const double* S, const double* U,
                          const double* rho_star);
void free_sources(Ctx* c);
bfvm_status launch_sources(Ctx* c, int p_next, bool renormed);
bfvm_status update_sources(Ctx* c, const double* pos, const double* vol, const double* S,
                           const double* U, const double* rho_star);
bfvm_status sync_source_counts(Ctx* c);

// Cell checking, sort keys and their sort on a plain stream (sources.cu),
// shared by the context's cell binning and bfvm_apply_sources_noalloc.
// A key is (voxel << kCellIdxBits) | cell index, unique per cell, so sorted
// keys give voxel order with cell-index order inside each voxel; padding
// keys (index >= n) are all ones and sort last.  The check ORs into *flag:
// 1 position outside [0, n_a dx], 2 volume, 4 rates, 8 rho*.
constexpr uint64_t kCellIdxBits = 31;
constexpr int kCellSortBlock = 2048;   // keys per shared-memory sort block
// z_origin / nz_global: the grid is the z-slab [z_origin, z_origin + nz)
// of a grid of nz_global layers (0 / nz for a whole grid); a cell belongs to
// the slab when its global voxel layer min(floor(p_z / dx), nz_global - 1)
// lies in it (else the check ORs 1), and its key holds the local voxel.
void launch_validate_cells(cudaStream_t st, int64_t n, int n_sub, const double* pos,
                           const double* vol, const double* S, const double* U,
                           const double* rs, double dx, int nx, int ny, int nz,
                           int z_origin, int nz_global, int* flag);
void launch_cell_keys(cudaStream_t st, int64_t n, int64_t n_pad, const double* pos, double dx,
                      int nx, int ny, int nz, int z_origin, int nz_global, uint64_t* keys);
// n_pad: a power of two >= kCellSortBlock; returns the number of launches
int64_t launch_sort_keys(cudaStream_t st, uint64_t* keys, int64_t n_pad);

// adjoint (adjoint.cu)
bfvm_status run_backward(Ctx* c, const double* g_final_dev, double* dD_dev,
                         double* dl_dev, double* dS_dev, double* dU_dev,
                         double* g0_dev);

// layout conversion between the caller's dense [s][z][y][x] and the pitched
// field (layout.cu)
// Device tables of the Dirichlet nodes (sweeps.cu): line-end values for the
// sweeps and the one-launch step's patch lists.  Nodes given as voxel,
// substrate, value and pitched field offset, one per (voxel, substrate).
bfvm_status build_node_tables(Ctx* c, const std::vector<int64_t>& vox,
                              const std::vector<int32_t>& sub, const std::vector<double>& val,
                              const std::vector<int64_t>& off);
bfvm_status copy_in_dense(Ctx* c, const void* src, bool on_device);
bfvm_status copy_out_dense(Ctx* c, void* dst, bool on_device);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace bfvm

struct bfvm_ctx {
    bfvm::Ctx impl;
};

namespace bfvm {

// Batched form: many contexts advanced by one launch per phase (batch.cu
// holds the ABI, sweeps.cu the kernels).
struct BatchImpl {
    std::vector<Ctx*> members;
    cudaStream_t stream = nullptr;
    int precision = 64;
    bool rescaled = false;
    int period = 1;
    int p = 0;                      // common rescale state of all members
    int max_n = 1;                  // longest line of any member and axis
    void* d_desc = nullptr;         // device array of per-member descriptors
    int2* d_tasks[3] = {nullptr, nullptr, nullptr};   // (member, 32-line block)
    int64_t n_tasks[3] = {0, 0, 0};
    int64_t* d_entry_prefix = nullptr;  // [members + 1] source entries
    int64_t n_entries = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_len = 0;
    int64_t launches = 0;
    std::string err;
    // Line-block shape of each axis' launch, chosen by measurement when the
    // batch is created (batch_tune): algo 0 = Thomas, one thread per line,
    // one warp per 32-line block; algo 1 = parallel cyclic reduction, one
    // warp per line (x lines of at most 128 voxels only); warps per CTA.
    int algo[3] = {0, 0, 0};
    int warps[3] = {8, 8, 8};
    double tune_ms[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};   // best Thomas, best PCR
    bool pcr_ok = false;          // every member's x lines are <= 128 voxels
    int pcr_e = 1;                // elements per lane of the PCR kernel (ceil(max nx / 32))
    double* d_pcr = nullptr;      // PCR stage tables of all members (FP64)
    float* d_pcr32 = nullptr;     // their FP32 hi/lo splits
    // One persistent launch per step (sweep_batch_step.cuh): warp pairs take
    // (axis, member-substrate group, 32-line block) tasks of all members.
    // one_launch: use it (where it fits); tables built at create.
    bool one_launch = false;      // the one-launch step is in use
    bool one_launch_ok = false;   // its tables exist (it fits this batch)
    int n_groups = 0;             // NS: member-substrate groups
    int n_btasks = 0;             // tasks of one step
    int64_t n_epi = 0;            // epilogue chunks of one step
    int b_slots = 0;              // column buffer slots (G x longest line in groups)
    int b_pairs = 0;              // warp pairs per CTA
    size_t b_smem = 0;            // dynamic shared memory per CTA
    void* d_members = nullptr;    // [period][members] member tables, one set per rescale state
    void* d_groups = nullptr;     // [3][NS] groups of the task list
    int64_t* d_epi_first = nullptr;   // [NS + 1] first epilogue chunk of each group
    int* d_gmem = nullptr;        // [NS] member of each group
    int* d_btask_first = nullptr; // [3 NS + 1]
    unsigned* d_bsched = nullptr; // claim, exit, done[3 NS], eclaim, shell_done[NS]
    int* d_err = nullptr;         // set when a bounded wait of the launch gave up
    int wait_test_polls = 0;      // > 0: waits cannot end (tests of the bounded waits)
};

bfvm_status batch_build(BatchImpl* b);
bfvm_status batch_set_shape(BatchImpl* b, int axis, int algo, int warps);
bfvm_status batch_launch_step(BatchImpl* b, int p, bool renorm);
void batch_free(BatchImpl* b);

}  // namespace bfvm

namespace bfvm {
// plain FP64 sweep along one axis, in -> out (sweeps.cu); dir_mode 0 step,
// 1 raw replay, 2 adjoint.  With out2, the warp-pair kernel writes its
// output to out2 as well where it runs, and sets c->dual_done.
bfvm_status launch_sweep_plain64(Ctx* c, int axis, const double* in, double* out,
                                 int dir_mode, double* out2 = nullptr);
}  // namespace bfvm
