/*
 * bfvm.h -- C ABI of the GB300 substrate transport step.
 *
 * The library advances the hybrid transport PDE of Eq. (1)
 *
 *     d rho/dt = D lap(rho) - lambda rho
 *                + sum_i delta(x - x_i) V_i (S_i (rho*_i - rho) - U_i rho)
 *
 * (element-wise over substrates) with the locally-one-dimensional (LOD)
 * implicit finite-volume scheme that the paper ports to the GPU
 * ("Using OpenACC programming model for PhysiCell", "Elements of
 * Parallelism": x-, y- and z-diffusion sweeps, Dirichlet conditions applied
 * on the device, AXPY-style line updates).  One step is
 *
 *   1. Dirichlet prologue: the outer voxel shell of every Dirichlet
 *      substrate is set to its value;
 *   2. x-solve: for every line along x, rho <- A_x^{-1} rho, where the line
 *      matrix has diagonal 1 + lambda dt/3 + c (ends) or 1 + lambda dt/3 + 2c
 *      (inside), off-diagonals -c, c = D dt / dx^2 (zero-flux faces); then
 *      the Dirichlet shell again;
 *   3. the same along y, then along z;
 *   4. cell sources: for each cell i in ascending index order, in its voxel v,
 *      rho_v <- (rho_v + dt (V_i/V_vox) S_i rho*_i) / (1 + dt (V_i/V_vox)(S_i+U_i)),
 *      V_vox = dx^3 (the delta term of Eq. 1, implicit in time).
 *
 * A cell at position p (micrometres, domain origin at 0) belongs to voxel
 * v_a = min(floor(p_a / dx), n_a - 1) on each axis a.
 *
 * Conventions shared by every call:
 *  - Field layout seen by callers: rho[s][z][y][x], x fastest, contiguous,
 *    n_sub * nz * ny * nx elements, element type double for precision 64 and
 *    float for precision 32.
 *  - Ownership: the context owns all of its device state (field,
 *    coefficient tables, binned cell data, checkpoints).  Buffers passed in
 *    are owned by the caller, are copied, and are never retained after the
 *    call returns.  With on_device = 1 a pointer is device memory of the
 *    context's device; the copy is ordered on the context's stream.  With
 *    on_device = 0 it is host memory and the call returns after the copy.
 *  - Errors: every call returns a bfvm_status; nothing is thrown across the
 *    ABI.  bfvm_last_error() gives a text for the last failure of a context.
 *    Arguments are checked on the host before any launch.  Kernels that wait
 *    on device flags give up after a bounded number of polls and report
 *    BFVM_ETIMEOUT instead of hanging.
 *  - Streams: cuda_stream is a cudaStream_t (NULL = the legacy default
 *    stream).  All work of a context is ordered on it.
 */
#ifndef BFVM_H
#define BFVM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BFVM_OK = 0,
    BFVM_EINVAL = 1,      /* bad argument (sizes, signs, non-finite, range) */
    BFVM_ENOMEM = 2,      /* a device or host allocation failed */
    BFVM_ECUDA = 3,       /* a CUDA runtime or driver call failed */
    BFVM_ESTATE = 4,      /* call not valid in the context's current state */
    BFVM_ETIMEOUT = 5,    /* a bounded device wait gave up */
    BFVM_ENONFINITE = 6   /* a NaN or Inf was found where it is not allowed */
} bfvm_status;

enum { BFVM_BC_ZERO_FLUX = 0, BFVM_BC_DIRICHLET = 1 };

typedef struct bfvm_ctx bfvm_ctx;
typedef struct bfvm_batch bfvm_batch;

/*
 * Create a simulation context (the device-side counterpart of the paper's
 * transfer-3D: allocate the field and the solver constants on the GPU once).
 *   nx, ny, nz    grid edges in voxels, each >= 1
 *   dx_um         voxel edge (micrometres), > 0; V_vox = dx^3
 *   dt_min        time step (minutes), > 0
 *   n_sub         number of substrates, >= 1
 *   D[n_sub]      diffusion coefficients (um^2/min), >= 0, finite
 *   lambda[n_sub] decay rates (1/min), >= 0, finite
 *   bc_kind[n_sub]  BFVM_BC_ZERO_FLUX or BFVM_BC_DIRICHLET (outer voxel
 *                 shell on all six faces held at bc_value)
 *   bc_value[n_sub] Dirichlet value (ignored for zero-flux), finite
 *   precision     64 (FP64 field and sweeps) or 32 (FP32 field and sweeps;
 *                 coefficient tables are still built in FP64, then rounded)
 *   cuda_stream   cudaStream_t for all of the context's work
 * The field starts at zero and there are no cells.  *out is set to NULL on
 * failure.  Host pointers are read during the call only.
 */
bfvm_status bfvm_create(bfvm_ctx** out, int32_t nx, int32_t ny, int32_t nz,
                        double dx_um, double dt_min, int32_t n_sub,
                        const double* D, const double* lambda,
                        const int32_t* bc_kind, const double* bc_value,
                        int32_t precision, void* cuda_stream);

/* Release every resource of the context (NULL is allowed). */
void bfvm_destroy(bfvm_ctx* ctx);

/*
 * Replace the whole field (paper: transfer-3D / translate-vector-to-array).
 *   rho  [n_sub][nz][ny][nx] of the context's element type, finite.
 * Resets any recorded forward run.
 */
bfvm_status bfvm_set_density(bfvm_ctx* ctx, const void* rho, int32_t on_device);

/*
 * Copy the field out (paper: translate-array-to-vector), same layout and
 * element type as bfvm_set_density.
 */
bfvm_status bfvm_get_density(bfvm_ctx* ctx, void* out, int32_t on_device);

/*
 * Set the cell agents that act as sources and sinks (the delta term of
 * Eq. 1).  All arrays are FP64, in cell-index order:
 *   pos[n][3]          position (um), each coordinate in [0, n_a * dx]
 *   vol[n]             volume V_i (um^3), > 0
 *   S[n][n_sub]        secretion rate (1/min), >= 0
 *   U[n][n_sub]        uptake rate (1/min), >= 0
 *   rho_star[n][n_sub] target density rho*_i, finite
 * n_cells = 0 removes all cells.  The cells are binned to voxels, stably
 * sorted by voxel (cell index order kept inside a voxel), and each voxel's
 * cells are composed, in index order and in FP64, into one affine map
 * rho <- alpha rho + beta per substrate.  Resets any recorded forward run.
 */
bfvm_status bfvm_set_cells(bfvm_ctx* ctx, int64_t n_cells, const double* pos,
                           const double* vol, const double* S, const double* U,
                           const double* rho_star, int32_t on_device);

/*
 * Dirichlet nodes inside the domain, e.g. vessels that hold a substrate at a
 * fixed level (an extension: the paper's models place such sources in the
 * tissue).  Node i holds substrate substrate[i] of voxel voxel[i]
 * (x + nx (y + ny z)) at value[i]: like the Dirichlet shell, the nodes are
 * set before the x-solve and after every solve (after the shell), so they
 * take part in each line solve and are overwritten after it; the cell
 * sources follow as usual.  Of two nodes on one voxel and substrate the
 * later one holds.  n_nodes = 0 removes all nodes.
 *   voxel[n]      int64, 0 <= voxel < nx ny nz
 *   substrate[n]  int32, 0 <= substrate < n_sub
 *   value[n]      FP64, finite
 * A node on a face of its substrate's Dirichlet shell is set after the
 * shell, so the solve of the line it ends takes the node's value there.
 * Arrays follow on_device like the other setters and are copied.  3-D
 * contexts only (BFVM_EINVAL for the 2-D variant).  In FP64 a step with
 * nodes is one node-fill launch plus option 8's one launch (node values
 * written after the x and y tasks that solve their lines and at the end of
 * the step); FP32 runs it one launch per axis with node fills between them.
 * A context with nodes cannot join a batch (BFVM_ESTATE).  Resets any
 * recorded forward run.
 */
bfvm_status bfvm_set_dirichlet_nodes(bfvm_ctx* ctx, int64_t n_nodes, const int64_t* voxel,
                                     const int32_t* substrate, const double* value,
                                     int32_t on_device);

/*
 * Move, resize or re-rate the cells of the last bfvm_set_cells without a
 * host round trip (an extension: the paper's agents move and grow on a
 * slower mechanics cadence than the diffusion steps, and names the host-side
 * cell handling its next bottleneck).  Same arrays and layout as
 * bfvm_set_cells, all DEVICE pointers, and n_cells must equal the count of
 * the last bfvm_set_cells (BFVM_EINVAL otherwise; BFVM_ESTATE if there were
 * no cells or a forward run is being recorded).
 * The cells are re-binned, re-sorted and their maps recomposed on the
 * context's stream, in tables sized by bfvm_set_cells: the call allocates
 * nothing, reads nothing back and returns at once.  The cells are checked
 * on the device: invalid ones (positions outside [0, n_a*dx], non-positive
 * volumes, negative or non-finite rates) make the next synchronising call
 * (bfvm_sync, bfvm_get_density to a host buffer) return BFVM_EINVAL, and
 * the field is then not valid; positions outside the domain are binned to
 * the nearest voxel meanwhile.
 */
bfvm_status bfvm_update_cells(bfvm_ctx* ctx, int64_t n_cells, const double* pos,
                              const double* vol, const double* S, const double* U,
                              const double* rho_star);

/* Advance n_steps >= 0 full steps (prologue, x, y, z, sources) on the
 * context's stream.  Asynchronous: errors of the kernels themselves surface
 * at the next synchronising call (bfvm_sync, bfvm_get_density with a host
 * pointer, bfvm_backward). */
bfvm_status bfvm_step(bfvm_ctx* ctx, int32_t n_steps);

/* Block until the context's stream is idle; reports device-side errors. */
bfvm_status bfvm_sync(bfvm_ctx* ctx);

/*
 * Enable (checkpoint_every >= 1) or disable (0) recording for the adjoint.
 * While enabled, each bfvm_step(n) stores the field at the start of steps
 * 0, k, 2k, ... of that call (ceil(n/k) fields of device memory) and
 * bfvm_backward then differentiates that call.
 */
bfvm_status bfvm_record(bfvm_ctx* ctx, int32_t checkpoint_every);

/*
 * Reverse mode of the last recorded bfvm_step(n) call.
 *   dL_drho_final  [n_sub][nz][ny][nx] FP64 gradient of the loss with
 *                  respect to the field after that call
 *   checkpoint_every  must equal the recorded interval (or 0 for "as
 *                  recorded")
 *   dD[n_sub], dlambda[n_sub]           FP64 outputs
 *   dS[n][n_sub], dU[n][n_sub]          FP64 outputs, cell-index order
 *   dL_drho0       optional (may be NULL) FP64 gradient with respect to the
 *                  field before the call
 * Every segment of k steps is replayed from its checkpoint; the adjoint of
 * each step runs the sources' adjoint, then the z, y, x solves (the line
 * matrices are symmetric), each after zeroing the adjoint of the Dirichlet
 * shell and of the Dirichlet nodes (a projection onto a fixed value does
 * not depend on its input).  The 2-D variant runs the y and x solves, each
 * with decay share lambda dt / 2.  Only FP64 contexts.  BFVM_ESTATE if
 * nothing was recorded.  Output pointers follow on_device like the input.
 */
bfvm_status bfvm_backward(bfvm_ctx* ctx, const double* dL_drho_final,
                          int32_t checkpoint_every, double* dD, double* dlambda,
                          double* dS, double* dU, double* dL_drho0,
                          int32_t on_device);

/* Text of the last failure on this context ("" if none; ctx may be NULL,
 * then the text of the last failed bfvm_create of this thread). */
const char* bfvm_last_error(const bfvm_ctx* ctx);

/* Name of a status code. */
const char* bfvm_status_string(int32_t status);

/*
 * Introspection, for tests and benchmarks.  info[16] receives:
 *  0 precision, 1 nx, 2 ny, 3 nz, 4 n_sub, 5 row pitch (elements),
 *  6 number of source voxels, 7 steps taken since create,
 *  8 sweep variant in use (0 plain, 1 rescaled), 9 rescale period,
 *  10 device kernel launches issued since create, 11 recorded steps,
 *  12 dimensions (3, or 2 for the 2-D variant), 13..15 reserved (0).
 */
bfvm_status bfvm_get_info(const bfvm_ctx* ctx, int64_t* info);

/*
 * Options (set before the first step; each returns BFVM_EINVAL for an
 * unknown key or value):
 *   key 1  sweep variant: 0 plain Thomas (3 flops per element per axis),
 *          1 rescaled Thomas (2 FMA per element per axis, FP64 only; the
 *          default for FP64)
 *   key 2  rescale period override (1..64; 0 = automatic)
 *   key 3  fuse cell sources into the z sweep: 0 no, 1 yes
 *   key 4  use CUDA graphs for bfvm_step: 0 no, 1 yes (default)
 *   key 5  per-kernel timing: 0 off (default), 1 each sweep and source
 *          launch is bracketed by CUDA events on the context's stream
 *          (bfvm_step then launches kernels one by one, without graphs)
 *   key 6  cap on the CTAs of the persistent sweeps (0 = one per SM, the
 *          default); small caps make every warp walk many line blocks
 *   key 7  sweep kernel: 0 warp pairs sharing each line buffer (the
 *          default), 1 one warp per line buffer
 *   key 8  with warp pairs (3-D grids; with Dirichlet nodes FP64 only):
 *          the x, y and z sweeps of a step, its Dirichlet shell, its nodes
 *          and its cell sources as one
 *          persistent launch whose warp pairs take (axis, substrate, 32-line
 *          block) tasks in order, a task starting once the previous axis of
 *          its substrate is complete.  1 (the default): where that launch
 *          gets at least as many warp pairs per SM as the per-axis launches
 *          (measured faster then for the FP64 forms; FP32 runs per axis); 2:
 *          wherever it fits; 0: one launch per axis
 *   key 10 dimensions: 3 (the default) or 2, the 2-D variant of the step
 *          (the paper ports BioFVM's 2-D diffusion too): for an nx x ny x 1
 *          grid, an x-solve and a y-solve per step, each line matrix with
 *          decay share lambda dt / 2; the Dirichlet shell is the outer layer
 *          of the four edges (the z layer is not a boundary); sources as in
 *          3-D with V_vox = dx^3.  Needs nz == 1; FP64 then runs the plain
 *          Thomas form (option 1 = 0).  2-D contexts can join a batch (it
 *          then runs the plain form for all members); dims cannot change
 *          while recording.
 *   key 11 split line solve of the plain form (the FP32 form, FP64 with
 *          key 1 = 0, and the 2-D variant): each line cut into segments
 *          solved in parallel, joined through the affine form of the two
 *          Thomas recurrences (three launches per axis).  1 (the default):
 *          for the 2-D variant and for lines too long for the shared-memory
 *          sweeps; 2: every plain-form sweep, the adjoint's included; 0: never
 *   key 9  test of the bounded device waits of key 8's launch: a value
 *          v > 0 makes every dependency wait unreachable and give up after
 *          v polls, so the next synchronising call reports BFVM_ETIMEOUT
 *          (results of such steps are not valid); 0 (the default) is normal
 *          operation
 */
bfvm_status bfvm_set_option(bfvm_ctx* ctx, int32_t key, int64_t value);

/*
 * Device time of the kernels timed under option 5, accumulated since the
 * last reset.  ms[5] (milliseconds) and counts[5] (launches) are host
 * arrays indexed by kind: 0 x sweep, 1 y sweep, 2 z sweep, 3 cell sources
 * and Dirichlet shell, 4 the x, y and z sweeps as one launch (option 8);
 * either may be NULL.  Synchronises the context's stream.  reset != 0 zeroes
 * the totals after reading them.
 */
bfvm_status bfvm_kernel_times(bfvm_ctx* ctx, double* ms, int64_t* counts, int32_t reset);

/*
 * Batched form: many independent contexts advanced together, one launch
 * per sweep phase over a flat list of line blocks of all members (captured
 * in a CUDA graph).  Members keep their own state; set and read them with
 * the single-context calls.  All members must use the same precision and
 * must not be stepped individually while the batch exists.
 */
/*
 * Batched form (an extension: the paper motivates many-run workflows such
 * as model calibration and parameter sweeps in "Introduction and
 * Motivation").  Create a batch over n_members existing contexts:
 *   members[i]  contexts of one device, all of the same precision, each at a
 *               rescale period boundary (fresh, or right after
 *               bfvm_set_density) and not recording, 3-D or 2-D (option 10;
 *               with any 2-D member the batch runs the plain Thomas form),
 *               without Dirichlet nodes and not z-slabs; the batch keeps
 *               pointers to them, so they must outlive it
 *   cuda_stream stream of the batched launches
 * Errors: BFVM_EINVAL (NULL pointers, n_members < 1), BFVM_ESTATE (mixed
 * precision, a member mid-period, recording, holding Dirichlet nodes or a
 * z-slab), BFVM_ENOMEM / BFVM_ECUDA.
 */
bfvm_status bfvm_batch_create(bfvm_batch** out, bfvm_ctx* const* members,
                              int32_t n_members, void* cuda_stream);
/* n_steps full steps of every member; asynchronous on the batch stream.
 * FP64 members share the shortest rescale period of the batch. */
bfvm_status bfvm_batch_step(bfvm_batch* batch, int32_t n_steps);
/* Block until the batch stream is idle; reports device-side errors. */
bfvm_status bfvm_batch_sync(bfvm_batch* batch);
/* Free the batch (the members stay valid). */
void bfvm_batch_destroy(bfvm_batch* batch);
const char* bfvm_batch_last_error(const bfvm_batch* batch);
/* info[8]: members, precision, rescaled (0/1), period, tasks per step over
 * the three sweeps, source entries, launches issued, current rescale state. */
bfvm_status bfvm_batch_info(const bfvm_batch* batch, int64_t* info);

/*
 * Line-block shape of the batched sweeps.  At bfvm_batch_create a built-in
 * autotuner times every candidate shape of each axis on scratch copies of
 * the members' fields (the fields themselves are not touched) and keeps the
 * fastest:
 *   algo 0  Thomas elimination, one thread per line, one warp per 32-line
 *           block, `warps` warps (2, 4 or 8, as far as the 32 x n line
 *           buffers fit in shared memory) per CTA;
 *   algo 1  parallel cyclic reduction (PCR) of the x lines, one warp per
 *           line holding it in registers, neighbours exchanged by warp
 *           shuffles, 4 or 8 warps per CTA; offered when no member's x line
 *           is longer than 128 voxels.  Its per-stage multipliers depend on
 *           the line matrix only and are built once, on the GPU, in FP64.
 * bfvm_batch_shape reads the chosen shape of an axis (0 x, 1 y, 2 z) and
 * ms[2] = the best measured time (ms per launch) of Thomas and of PCR
 * (-1 where not measured).  bfvm_batch_set_shape forces a shape (EINVAL
 * for an unsupported one).  Both give the same results up to rounding.
 */
bfvm_status bfvm_batch_shape(const bfvm_batch* batch, int32_t axis, int32_t* algo,
                             int32_t* warps, double* ms);
bfvm_status bfvm_batch_set_shape(bfvm_batch* batch, int32_t axis, int32_t algo, int32_t warps);

/*
 * Options of a batch (each returns BFVM_EINVAL for an unknown key or value):
 *   key 1  1: each step of the batch as one persistent launch whose warp
 *          pairs take (axis, member substrate, 32-line block) tasks of all
 *          members in order, a task starting once the previous axis of its
 *          member's substrate is complete, followed in the same launch by
 *          the members' Dirichlet shells and cell sources (the default where
 *          its column buffers fit in shared memory; BFVM_EINVAL otherwise);
 *          0: one launch per sweep phase with the tuned line-block shapes
 *   key 2  test of the bounded device waits of key 1's launch: v > 0 makes
 *          every dependency wait unreachable and give up after v polls, so
 *          bfvm_batch_sync reports BFVM_ETIMEOUT (results of such steps are
 *          not valid); 0 (the default) is normal operation
 */
bfvm_status bfvm_batch_set_option(bfvm_batch* batch, int32_t key, int64_t value);

/*
 * One grid decomposed along z into slabs, one context per slab (an
 * extension: the paper names an MPI+X decomposition of the domain as its
 * way to larger problems, "Introduction and Motivation" and "Future Work").
 * The slabs together compute exactly the step of the whole grid (up to
 * rounding): the x and y lines lie inside a slab; each z line is solved by
 * the Thomas algorithm of the whole line, split into the slabs' segments
 * through the affine form of its two recurrences, with one exchange of one
 * value per z line and substrate after the forward and after the backward
 * pass.
 *
 * Create slab `slab` of n_slabs: the grid is nx x ny x z_starts[n_slabs],
 * slab j holding the global layers [z_starts[j], z_starts[j+1]) (z_starts[0]
 * = 0, every slab at least one layer).  The other arguments are those of
 * bfvm_create; the context is FP64 in the plain Thomas form.  Its field is
 * the slab's part of the grid, [n_sub][nz_j][ny][nx] with nz_j its layer
 * count, set and read with bfvm_set_density / bfvm_get_density.  Its cells
 * are given in grid coordinates (positions in [0, n_a dx] of the whole
 * grid); every cell's voxel layer must lie in the slab (BFVM_EINVAL
 * otherwise).  A slab context rejects bfvm_step, recording for the adjoint,
 * Dirichlet nodes, options 1, 2, 8 and 10 and batches (BFVM_ESTATE).
 */
bfvm_status bfvm_create_slab(bfvm_ctx** out, int32_t nx, int32_t ny, int32_t n_slabs,
                             const int32_t* z_starts, int32_t slab, double dx_um,
                             double dt_min, int32_t n_sub, const double* D,
                             const double* lambda, const int32_t* bc_kind,
                             const double* bc_value, void* cuda_stream);

/*
 * One step of a slab, in three calls with two gathers between them.  The
 * first two write one FP64 value per z line and substrate to the caller's
 * device buffer send[n_sub][ny][nx]; the caller gathers the send buffers of
 * all slabs, in slab order, into one device array gathered[n_slabs][n_sub]
 * [ny][nx] (e.g. an all-gather across ranks, after the context's stream has
 * finished the call) and passes it to the next call.  Both buffers stay the
 * caller's; the calls read or write them on the context's stream.
 *   bfvm_slab_forward   the x and y sweeps with their Dirichlet handling,
 *                       then the z forward elimination of the slab's
 *                       segment from a zero incoming value; send = its last
 *                       values
 *   bfvm_slab_backward  the segment's incoming forward value from the
 *                       gathered values of the slabs below, then its back
 *                       substitution from a zero incoming value; send = its
 *                       first values
 *   bfvm_slab_finish    the incoming value from the gathered values of the
 *                       slabs above, the z solution, the grid's Dirichlet
 *                       shell within the slab and the slab's cell sources
 * All three are asynchronous.  BFVM_ESTATE on a context that is not a slab,
 * BFVM_EINVAL for NULL buffers.
 */
bfvm_status bfvm_slab_forward(bfvm_ctx* ctx, double* send);
bfvm_status bfvm_slab_backward(bfvm_ctx* ctx, const double* gathered, double* send);
bfvm_status bfvm_slab_finish(bfvm_ctx* ctx, const double* gathered);

/*
 * Measured FP64 fused multiply-add rate of the current device (the paper
 * has no counterpart: it is the denominator of the FP64-pipe roofline of
 * the FP64 sweeps, which spend two FMAs per element and axis).  One CTA of
 * warps_per_sm (1..32) warps per SM; every thread runs `chains` (1, 2, 4 or
 * 8) independent chains x <- a x + b for 8 * iters (iters 1..2^24) rounds;
 * the launch is timed with CUDA events on cuda_stream.
 *   fma_per_second  out: FMAs (lane operations) per second
 *   elapsed_ms      out, may be NULL: the timed launch's duration
 * Allocates and frees a small output buffer; synchronises cuda_stream.
 * Errors: BFVM_EINVAL (arguments), BFVM_ECUDA; text via bfvm_last_error(NULL).
 */
bfvm_status bfvm_fp64_fma_rate(int32_t warps_per_sm, int32_t chains, int64_t iters,
                               void* cuda_stream, double* fma_per_second, double* elapsed_ms);

/*
 * Allocation-free variant of the cell source/uptake update.  The paper has
 * no counterpart: it exists for callers that must not allocate device
 * memory, such as host loops driving many small simulations (cudaMalloc and
 * cudaFree stall, and cudaFree synchronises the whole device) or programs
 * whose memory manager owns all device memory.
 *
 * Applies, to the caller's dense FP64 device field rho[n_sub][nz][ny][nx]
 * (in place), the same update as the source part of bfvm_step: every cell,
 * in ascending index order within its voxel, does
 *   rho_v <- (rho_v + dt (V_i/dx^3) S_i rho*_i) / (1 + dt (V_i/dx^3)(S_i+U_i)).
 * pos, vol, S, U, rho_star are device arrays laid out as in bfvm_set_cells.
 * Their sizes are taken on trust: rho must hold n_sub*nz*ny*nx doubles,
 * pos 3*n_cells, vol n_cells, and S, U, rho_star n_cells*n_sub each, all on
 * the current device (the Python binding checks shapes, dtypes and devices
 * before calling).
 * It allocates nothing: its only scratch (the sort keys of at most 262,144
 * cells plus a check flag, about 2 MB) is a fixed device array that every
 * GPU loading this library holds until the process exits.
 *  - n_cells > 262,144: BFVM_EINVAL with an explanatory text, nothing runs.
 *  - Bad sizes or cells (positions outside [0, n_a*dx], non-positive
 *    volumes, negative or non-finite rates): BFVM_EINVAL; the field is
 *    untouched.  Every call synchronises cuda_stream once, to read the cell
 *    check back before the update is launched.
 *  - Errors are reported by bfvm_last_error(NULL).
 *  - The first call on a device looks up the scratch array's device address
 *    (once per device, with that device current) and keeps it; make that
 *    first call before any stream capture.  The kept address belongs to the
 *    device's primary context: do not call this entry point again in a
 *    process after cudaDeviceReset on that device.
 *  - All calls on one device share the scratch: calls whose GPU work can
 *    overlap (different streams without ordering) race; order them on one
 *    stream.  Each call rewrites every scratch word it reads.
 */
bfvm_status bfvm_apply_sources_noalloc(double* rho, int32_t nx, int32_t ny, int32_t nz,
                                       int32_t n_sub, double dx_um, double dt_min,
                                       int64_t n_cells, const double* pos,
                                       const double* vol, const double* S,
                                       const double* U, const double* rho_star,
                                       void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* BFVM_H */
