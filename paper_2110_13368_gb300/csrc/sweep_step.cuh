// The three sweeps of one step (any form and precision) as one persistent
// launch (included by sweeps.cu after sweep_pair.cuh, whose PairSweeper it
// drives).
//
// Why: one pair of warps sweeps a 32-line block in one phase (the forward
// elimination of block k+1 next to the back substitution of block k).  A
// separate launch per axis gives each pair only a few blocks, and every
// launch pays a phase in which one warp of each pair has nothing to do (the
// first block's forward and the last block's back substitution), plus the
// tail where the pairs that drew one block more than the rest finish
// alone.  Here the pairs keep their pipeline running across axes and
// substrates, so that cost is paid once per step.
//
// Tasks: (axis a, substrate s, block j) with blocks of 32 lines of the line
// set of (a, s) (lines entirely on a Dirichlet shell are not in the set;
// blocks never straddle substrates), numbered axis-major: all x tasks of
// substrate 0, of substrate 1, ..., then the y tasks, then the z tasks.
// task_first[a * n_sub + s] is the first task of (a, s).
//
// Dependencies: a task of (a, s) with a > 0 reads lines that every task of
// (a - 1, s) writes, so it starts only when done[a - 1][s] (tasks of
// (a - 1, s) completed) reaches their count (an axis without tasks is
// skipped: the nearest earlier axis of s that has tasks counts).  With several substrates the
// order above leaves the tasks of the other substrates between a task and
// its dependencies, so the wait is normally over before it starts.
//
// Scheduling: each pair's F warp claims tasks from a counter (atomicAdd),
// one task ahead of the one it eliminates, so tasks are claimed in order by
// pairs that are running, and a claimed task only waits on tasks with
// smaller numbers.  A pair never blocks while it holds a started task that
// another task needs: when the task F is to start next has incomplete input,
// B back-substitutes its current task on its own (no pair barriers), signals
// its completion, and only then does F wait.  The smallest unfinished task
// is therefore never stuck (if it is started, its pair runs; if it is only
// claimed, its pair's F is waiting on smaller, finished tasks), and every
// wait ends.  Waits are still bounded (kMaxPolls polls): on expiry the kernel sets
// the error flag (reported as BFVM_ETIMEOUT by the next synchronising call)
// and carries on.
//
// Memory ordering: B makes its stores visible (fence) before lane 0 adds to
// done[a][s]; F reads done with ld.acquire and then every lane executes an
// acquire fence, so the copies that follow (cp.async through L1) see the
// other SMs' writes and no L1 line left from an earlier task of this SM.
//
// Epilogue: every warp that runs out of sweep tasks takes chunks of the
// Dirichlet shell fill and of the cell sources (step_epilogue), so both run
// in the same launch, next to the last sweep tasks.
//
// The counters (claim, exit, done, epilogue) are zero at every launch: the
// last CTA to finish resets them, and the next launch is ordered after this
// one on the stream.
#pragma once

namespace bfvm {
namespace persistent {

struct StepSched {
    unsigned* claim;        // [1] next task to hand out
    unsigned* exit_count;   // [1] CTAs that have finished
    unsigned* done;         // [3 * n_sub] completed tasks per (axis, substrate)
    const int* task_first;  // [3 * n_sub + 1] first task of (axis, substrate)
    int* err;               // set to 1 when a dependency wait gave up
    int n_sub;
    int n_tasks;
    unsigned max_polls;     // polls before a wait gives up (kMaxPolls)
    unsigned extra_need;    // 0; 1 only to test the give-up path (no wait can end)
    // epilogue of the step (after every z task of a substrate): the
    // Dirichlet shell, then the cell sources, in chunks of kEpiChunk
    unsigned* eclaim;       // [1] next epilogue chunk
    unsigned* shell_done;   // [n_sub] completed shell and node chunks of each substrate
    int n_epi_chunks;       // over all substrates
    // Dirichlet nodes (the kernel's NODES form): the nodes on the lines of
    // each x and y task, written after the task's outputs, and every node by
    // substrate, written by the epilogue's node chunks (after the substrate's
    // shell, before its sources)
    const int* node_task_first;   // [n_tasks + 1]
    const NodePatch* node_patch;
    const int* node_sfirst;       // [n_sub + 1]
    const NodePatch* node_epi;
};

// Everything the epilogue reads: grid, the scales of state p + 1 (null when
// the step renormalises: plain values) and the composed cell maps.
template <typename T>
struct EpiArgs {
    T* field;
    int nx, ny, nz;
    int64_t pitch, L;
    const double* sc;       // [s][L] scales of state p + 1, or null
    int64_t n_seg;          // occupied voxels; entry g * n_sub + s is voxel g, substrate s
    const int64_t* d_nseg;  // or null; else the exact count, n_seg being an upper bound
    const int64_t* off;     // field offset of each (voxel, substrate) entry
    const double* alpha;
    const double* beta;
    const int32_t* vox;     // voxel x + nx (y + ny z)
    const int32_t* sub;
    int zf;                 // batched step: z planes on the boundary (0: the 2-D variant)
};

constexpr int kEpiUnroll = 8;                  // independent elements per lane
constexpr int kEpiChunk = 32 * kEpiUnroll * 2;  // elements per claimed chunk (2 rounds)
constexpr int kNodeUnroll = 4;                 // nodes per lane of an epilogue node chunk
constexpr int kNodeChunk = 32 * kNodeUnroll;

// Epilogue chunks, substrate by substrate: the shell chunks of s (Dirichlet
// substrates only), then its source chunks (kEpiChunk occupied voxels each).
__host__ __device__ inline int64_t epi_shell_chunks(int nx, int ny, int nz)
{
    const int64_t per = 2 * ((int64_t)nx * ny + (int64_t)nx * nz + (int64_t)ny * nz);
    return (per + kEpiChunk - 1) / kEpiChunk;
}
__host__ __device__ inline int64_t epi_src_chunks(int64_t n_seg)
{
    return (n_seg + kEpiChunk - 1) / kEpiChunk;
}

// The same for a grid whose z planes are boundary faces (zf != 0: the 3-D
// shell) or not (zf == 0: the 2-D variant's four edges, the enumeration of
// shell_voxel without its z-plane part)
__host__ __device__ inline int64_t shell_count_z(int nx, int ny, int nz, int zf)
{
    return 2 * ((zf ? (int64_t)nx * ny : 0) + (int64_t)nx * nz + (int64_t)ny * nz);
}
__host__ __device__ inline int64_t epi_shell_chunks_z(int nx, int ny, int nz, int zf)
{
    return (shell_count_z(nx, ny, nz, zf) + kEpiChunk - 1) / kEpiChunk;
}

// about 2^21 polls with a 128 ns back-off: well over a second
constexpr unsigned kMaxPolls = 1u << 21;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

struct TaskRef {
    int a, s, j;   // axis, substrate, block within (a, s)
};

__device__ __forceinline__ TaskRef decode_task(const int* tf, int n_sub, int t)
{
    int i = 0;
    const int last = 3 * n_sub;
    while (i + 1 < last && t >= tf[i + 1]) ++i;
    TaskRef r;
    r.a = i / n_sub;
    r.s = i % n_sub;
    r.j = t - tf[i];
    return r;
}

// Completion counter that a task of axis a (0..2; 3 = the epilogue) of
// substrate s waits on: that of the nearest earlier axis of s that has
// tasks (on a Dirichlet substrate an axis can have none, e.g. when another
// extent is at most 2), or -1 when no earlier axis has any.
__device__ __forceinline__ int dep_index(const int* tf, int n_sub, int a, int s)
{
    for (int b = a - 1; b >= 0; --b) {
        const int i = b * n_sub + s;
        if (tf[i + 1] > tf[i]) return i;
    }
    return -1;
}

// F warp: next task number (n_tasks when none is left)
__device__ __forceinline__ int claim_task(const StepSched& Q, int lane)
{
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(Q.claim, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    return t < (unsigned)Q.n_tasks ? (int)t : Q.n_tasks;
}

// F warp: is the input of task r complete?  (no waiting)
__device__ __forceinline__ bool task_ready(const StepSched& Q, const int* tf, TaskRef r, int lane)
{
    const int i = dep_index(tf, Q.n_sub, r.a, r.s);
    if (i < 0) return true;
    const unsigned need = (unsigned)(tf[i + 1] - tf[i]) + Q.extra_need;
    int ok = 0;
    if (lane == 0) ok = ld_acquire_u32(Q.done + i) >= need;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) fence_acq_rel_gpu();
    return ok != 0;
}

// F warp: wait (bounded) until the input of task r is complete
__device__ __forceinline__ void task_wait(const StepSched& Q, const int* tf, TaskRef r, int lane)
{
    const int i = dep_index(tf, Q.n_sub, r.a, r.s);
    if (i < 0) return;
    const unsigned need = (unsigned)(tf[i + 1] - tf[i]) + Q.extra_need;
    if (lane == 0) {
        unsigned polls = 0;
        while (ld_acquire_u32(Q.done + i) < need) {
            if (++polls > Q.max_polls) {
                atomicExch(Q.err, 1);
                break;
            }
            __nanosleep(128);
        }
    }
    __syncwarp();
    fence_acq_rel_gpu();
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// B warp: all of task r's outputs are stored; publish its completion (each
// lane's release fence orders its stores before lane 0's count)
__device__ __forceinline__ void task_done(const StepSched& Q, TaskRef r, int lane)
{
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) atomicAdd(Q.done + r.a * Q.n_sub + r.s, 1u);
}

// Line of this lane in task r (padding lanes past the set's end repeat its
// last line and are not stored)
template <typename T, int AXIS, int MODE>
__device__ __forceinline__ Line task_line(const SweepArgs<T>& A, const LineSet& S,
                                          const int64_t* fs, TaskRef r, int lane)
{
    const int64_t hi = fs[r.s + 1];
    int64_t line = fs[r.s] + (int64_t)r.j * 32 + lane;
    const bool valid = line < hi;
    if (!valid) line = hi - 1;
    Line L = make_line<T, AXIS, MODE>(A, S, fs, line);
    L.valid = valid;
    return L;
}

// A task's lines in two halves: issue_line() computes the integer part and
// issues the few global reads a line needs (the Dirichlet value's scales of
// the other axes and of this axis' two ends, the renormalising inverse
// scales), finish_line() does the arithmetic on them.  F issues the reads
// of its next task before it eliminates the current one and finishes them
// after, so their latency overlaps the elimination.
struct LinePre {
    int64_t base;
    int s;
    bool valid, dir;
    double v, v1, sa, sb, se0, se1, ia, ib;   // v, v1: input values of the two ends
};

// NODES: a Dirichlet node may sit at either end of the line (its value
// then replaces the boundary value there)
template <typename T, int AXIS, int MODE, bool NODES = false>
__device__ __forceinline__ LinePre issue_line(const SweepArgs<T>& A, const LineSet& S,
                                              const int64_t* fs, const int* bck,
                                              const double* bcv, TaskRef r, int lane)
{
    LinePre P;
    const int64_t hi = fs[r.s + 1];
    int64_t t = (int64_t)r.j * 32 + lane;
    P.valid = fs[r.s] + t < hi;
    if (!P.valid) t = hi - 1 - fs[r.s];
    const int s = r.s;
    P.s = s;
    const int ca = S.cnt_a[s];
    const int a = S.lo_a[s] + (int)(t % ca);
    const int b = S.lo_b[s] + (int)(t / ca);
    int ox = 0, oy = 0, oz = 0;
    if (AXIS == 0) {
        oy = a; oz = b;
        P.base = (((int64_t)s * A.nz + oz) * A.ny + oy) * A.pitch;
    } else if (AXIS == 1) {
        ox = a; oz = b;
        P.base = (((int64_t)s * A.nz + oz) * A.ny) * A.pitch + ox;
    } else {
        ox = a; oy = b;
        P.base = ((int64_t)s * A.nz * A.ny + oy) * A.pitch + ox;
    }
    P.dir = bck[s] == BFVM_BC_DIRICHLET;
    P.v = bcv[s];
    P.v1 = P.v;
    if (NODES && P.dir) end_values(A.ends, full_line<T, AXIS>(A, s, ox, oy, oz), bcv[s], P.v, P.v1);
    P.sa = P.sb = P.se0 = P.se1 = P.ia = P.ib = 1.0;
    if (MODE >= 1 && P.dir) {
        const int64_t row = (int64_t)s * A.L;
        if (AXIS == 0) {
            P.sa = A.sc_p[row + A.off_y + oy];
            P.sb = A.sc_p[row + A.off_z + oz];
        } else if (AXIS == 1) {
            P.sa = A.sc_p1[row + A.off_x + ox];
            P.sb = A.sc_p[row + A.off_z + oz];
        } else {
            P.sa = A.sc_p1[row + A.off_x + ox];
            P.sb = A.sc_p1[row + A.off_y + oy];
        }
        P.se0 = A.sc_p[row + A.axis_off];
        P.se1 = A.sc_p[row + A.axis_off + A.n - 1];
    }
    if (MODE == 2 && AXIS == 2) {
        const int64_t row = (int64_t)s * A.L;
        P.ia = A.isc_p1[row + A.off_x + ox];
        P.ib = A.isc_p1[row + A.off_y + oy];
    }
    return P;
}

template <int MODE, bool NODES = false>
__device__ __forceinline__ Line finish_line(const LinePre& P)
{
    Line L;
    L.base = P.base;
    L.s = P.s;
    L.valid = P.valid;
    L.dir = P.dir;
    if (MODE >= 1 && NODES) {
        L.end0 = (P.v * P.sa * P.sb) * P.se0;
        L.end1 = (P.v1 * P.sa * P.sb) * P.se1;
    } else if (MODE >= 1) {
        const double kline = P.v * P.sa * P.sb;
        L.end0 = kline * P.se0;
        L.end1 = kline * P.se1;
    } else {
        L.end0 = P.v;
        L.end1 = NODES ? P.v1 : P.v;
    }
    L.inv_other = P.ia * P.ib;
    return L;
}

// The kernel's shared copies of the coefficients, [s][L] per table: the
// forward and backward coefficients (fa / fb of the rescaled form, r / cr of
// the plain form) and, for the FP32 plain form, their low parts.
template <typename T>
struct CoefTabs {
    const T* a;
    const T* b;
    const T* a_lo;
    const T* b_lo;
};

// Coefficient rows of substrate s on this axis from the shared tables
// (every lane of a task has the same s, so each read is a broadcast); the
// plain form's off-diagonal c and the output scales of a renormalising z
// sweep from global memory
template <typename T, int AXIS, int MODE>
__device__ __forceinline__ CoefRow<T> step_coef_row(const SweepArgs<T>& A, const CoefTabs<T>& K,
                                                    int s)
{
    CoefRow<T> C;
    const int64_t row = (int64_t)s * A.L + A.axis_off;
    C.a = K.a + row;
    C.b = K.b + row;
    C.a_lo = K.a_lo + row;
    C.b_lo = K.b_lo + row;
    C.o = A.isc_p1 + row;
    C.c = (T)0;
    C.c_lo = (T)0;
    if (MODE == 0) {
        C.c = A.cvec[s * 3 + AXIS];
        if (sizeof(T) == 4) C.c_lo = A.cvec_lo[s * 3 + AXIS];
    }
    return C;
}

template <typename T>
__device__ __forceinline__ int64_t axis_stride(const SweepArgs<T>& A, int axis)
{
    return axis == 0 ? 1 : (axis == 1 ? A.pitch : (int64_t)A.ny * A.pitch);
}

// F: copies and forward elimination of task r with slot parity q; solo:
// the whole task on its own, else next to B's back substitution with
// `iters` pair-barrier meetings.  Returns the chain value of the last
// element (handed to B).
template <typename T, int AXIS, int MODE>
__device__ __forceinline__ T f_task(const SweepArgs<T>& A, const Line& L, T* field,
                                    const CoefTabs<T>& K, T* W, int ns, int lane, int bar_id,
                                    int64_t* rbF, int q, bool solo, int iters)
{
    constexpr int G = Groups<T>::G;
    PairSweeper<T, AXIS, MODE> sw{A, W, field, field, axis_stride(A, AXIS), A.n, ns, lane, bar_id};
    const CoefRow<T> C = step_coef_row<T, AXIS, MODE>(A, K, L.s);
    __syncwarp();
    rbF[lane] = L.base;
    __syncwarp();
    int64_t rv[G];
    sw.load_rows(rbF, rv);
    T prev;
    if (solo) {
        const int gcount = (A.n + G - 1) / G;
        for (int g = 0; g < gcount; ++g) {
            if (q) sw.template copy_group<1>(L, rbF, g);
            else sw.template copy_group<0>(L, rbF, g);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        prev = q ? sw.template f_solo<1>(L, C) : sw.template f_solo<0>(L, C);
    } else {
        prev = q ? sw.template f_block<1>(L, C, rbF, rv, iters)
                 : sw.template f_block<0>(L, C, rbF, rv, iters);
        cp_async_wait<0>();
    }
    return prev;
}

// B: back substitution of task r (parity q) from chain value x, with or
// without F next to it.  The line bases (-1 for padding lanes) and the
// substrate come from F through shared memory (rbB, hs): F built them when
// it eliminated the task.  `rel` publishes the task's completion.
template <typename T, int AXIS, int MODE, typename Rel>
__device__ __forceinline__ void b_task(const SweepArgs<T>& A, const LineSet& S,
                                       const int64_t* fs, const int* bck, const double* bcv,
                                       T* field, const CoefTabs<T>& K, T* W, int ns, int lane,
                                       int bar_id, TaskRef r, const int64_t* rbB, const int* hs,
                                       int q, T x, bool paired, int iters, const Rel& rel)
{
    constexpr int G = Groups<T>::G;
    PairSweeper<T, AXIS, MODE> sw{A, W, field, field, axis_stride(A, AXIS), A.n, ns, lane, bar_id};
    Line L;
    const int64_t hb = rbB[lane];
    L.valid = hb >= 0;
    L.base = L.valid ? hb : 0;
    L.s = hs[lane];
    L.dir = false;
    L.end0 = L.end1 = 0.0;
    L.inv_other = 1.0;
    if (MODE == 2) L.inv_other = finish_line<MODE>(issue_line<T, AXIS, MODE>(A, S, fs, bck, bcv, r, lane)).inv_other;
    const CoefRow<T> C = step_coef_row<T, AXIS, MODE>(A, K, L.s);
    int64_t rv[G];
    sw.load_rows(rbB, rv);
    if (q) sw.template b_block<1>(L, C, x, rbB, rv, paired, iters, rel);
    else sw.template b_block<0>(L, C, x, rbB, rv, paired, iters, rel);
}

// Shell voxels of one Dirichlet substrate, enumerated as z planes (2 nx ny),
// y rows of the other planes (2 nx nz), x columns (2 ny nz); overlaps are
// written twice with the same value.
template <typename T>
__device__ __forceinline__ int64_t shell_count(const EpiArgs<T>& E)
{
    return 2 * ((int64_t)E.nx * E.ny + (int64_t)E.nx * E.nz + (int64_t)E.ny * E.nz);
}

template <typename T>
__device__ __forceinline__ void shell_voxel(const EpiArgs<T>& E, int s, double v, int64_t t64)
{
    // 32-bit index arithmetic (64-bit division is far slower): the kernels
    // that run this epilogue hold a whole line of every axis in one shared
    // column buffer, so no extent exceeds a few thousand voxels and the shell
    // has far fewer than 2^31 voxels
    const int nx = E.nx, ny = E.ny, nz = E.nz;
    const int fz = 2 * nx * ny, fy = 2 * nx * nz;
    int t = (int)t64;
    int x, y, z;
    if (t < fz) {
        const int q = t / nx;
        x = t - q * nx; y = q % ny; z = (q / ny) ? nz - 1 : 0;
    } else if ((t -= fz) < fy) {
        const int q = t / nx;
        x = t - q * nx; z = q % nz; y = (q / nz) ? ny - 1 : 0;
    } else {
        t -= fy;
        const int q = t / ny;
        y = t - q * ny; z = q % nz; x = (q / nz) ? nx - 1 : 0;
    }
    if (E.sc) {
        const double* q = E.sc + (int64_t)s * E.L;
        v = v * (__ldg(q + x) * __ldg(q + E.nx + y) * __ldg(q + E.nx + E.ny + z));
    }
    E.field[(((int64_t)s * E.nz + z) * E.ny + y) * E.pitch + x] = (T)v;
}

// Wait (bounded) until counter p reaches need; lane 0 polls, then every
// lane executes an acquire fence.
__device__ __forceinline__ void wait_count(const StepSched& Q, const unsigned* p, unsigned need,
                                           int lane)
{
    if (lane == 0) {
        unsigned polls = 0;
        while (ld_acquire_u32(p) < need) {
            if (++polls > Q.max_polls) {
                atomicExch(Q.err, 1);
                break;
            }
            __nanosleep(128);
        }
    }
    __syncwarp();
    fence_acq_rel_gpu();
}

// Epilogue node chunks of substrate s (NODES form): kNodeChunk nodes each
__device__ __forceinline__ int epi_node_chunks(const StepSched& Q, int s)
{
    return (Q.node_sfirst[s + 1] - Q.node_sfirst[s] + kNodeChunk - 1) / kNodeChunk;
}

// A warp with no sweep task left takes epilogue chunks, claimed in order:
// for each substrate s, the shell chunks of s once every task of the last
// swept axis of s is complete, then (NODES) its node chunks once the shell
// of s is complete too (a node overrides the shell), then the source chunks
// of s once the shell and the nodes of s are complete (a cell may sit in a
// shell voxel or on a node).  A chunk waits only on sweep tasks and on
// earlier chunks that never wait on it, and a warp acquires each completion
// at most once.
template <typename T, bool NODES = false>
__device__ __forceinline__ void step_epilogue(const StepSched& Q, const EpiArgs<T>& E,
                                              const int* tf, const int* bck, const double* bcv,
                                              int lane)
{
    const int n_sub = Q.n_sub;
    const int64_t per = shell_count(E);
    const int sh_chunks = (int)epi_shell_chunks(E.nx, E.ny, E.nz);
    const int src_chunks = (int)epi_src_chunks(E.n_seg);
    const int64_t n_seg = E.d_nseg ? *E.d_nseg : E.n_seg;   // written before this launch
    unsigned long long got = 0ull;   // bit s: sweeps of s acquired; bit 32 + s: shell of s
    for (;;) {
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(Q.eclaim, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= (unsigned)Q.n_epi_chunks) return;
        int s = 0, k = (int)c;
        for (; s < n_sub; ++s) {
            const int here = (bck[s] == BFVM_BC_DIRICHLET ? sh_chunks : 0) +
                             (NODES ? epi_node_chunks(Q, s) : 0) + src_chunks;
            if (k < here) break;
            k -= here;
        }
        const bool dir = bck[s] == BFVM_BC_DIRICHLET;
        const bool mask_ok = s < 32;
        const bool shell = dir && k < sh_chunks;
        const int nch = NODES ? epi_node_chunks(Q, s) : 0;
        // node chunk kn of s (NODES), else -1
        const int kn = (NODES && !shell && k - (dir ? sh_chunks : 0) < nch)
                           ? k - (dir ? sh_chunks : 0) : -1;
        if (NODES && kn >= 0) {
            if (!(mask_ok && ((got >> s) & 1ull))) {
                const int i = dep_index(tf, n_sub, 3, s);
                if (i >= 0) wait_count(Q, Q.done + i, (unsigned)(tf[i + 1] - tf[i]) + Q.extra_need, lane);
                if (mask_ok) got |= 1ull << s;
            }
            if (dir) wait_count(Q, Q.shell_done + s, (unsigned)sh_chunks + Q.extra_need, lane);
            // the node values after the step's sweeps and shell (scales of
            // state p + 1, or plain values)
            const int lo = Q.node_sfirst[s] + kn * kNodeChunk;
            const int hi = min(Q.node_sfirst[s + 1], lo + kNodeChunk);
            NodePatch e[kNodeUnroll];
#pragma unroll
            for (int u = 0; u < kNodeUnroll; ++u)
                if (lo + lane + 32 * u < hi) e[u] = Q.node_epi[lo + lane + 32 * u];
#pragma unroll
            for (int u = 0; u < kNodeUnroll; ++u) {
                if (lo + lane + 32 * u >= hi) continue;
                double v = e[u].v;
                if (E.sc) {
                    const double* q = E.sc + (int64_t)s * E.L;
                    v = v * (__ldg(q + e[u].x) * __ldg(q + E.nx + e[u].y) *
                             __ldg(q + E.nx + E.ny + e[u].z));
                }
                E.field[e[u].off] = (T)v;
            }
            fence_acq_rel_gpu();
            __syncwarp();
            if (lane == 0) atomicAdd(Q.shell_done + s, 1u);
            continue;
        }
        // a source chunk reads its entries (field offsets, the composed
        // maps, the scale of each voxel) before it waits for the sweeps:
        // none of them depends on the step, so only the field's gather and
        // update are left for after the wait (a warp that claims a chunk of
        // the last swept substrate waits for its last z tasks)
        constexpr int R = kEpiChunk / 32;
        int64_t o[R];
        double a[R], b[R];
        if (!shell) {
            const int kk = (dir ? k - sh_chunks : k) - nch;
            const int64_t lo = (int64_t)kk * kEpiChunk;
            const int64_t hi = min(n_seg, lo + kEpiChunk);
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int64_t g = lo + lane + 32 * u;
                o[u] = -1;
                if (g < hi) {
                    const int64_t e = g * n_sub + s;
                    o[u] = __ldg(E.off + e);
                    a[u] = __ldg(E.alpha + e);
                    b[u] = __ldg(E.beta + e);
                    if (E.sc) {
                        const int32_t vv = __ldg(E.vox + e);
                        const int x = vv % E.nx;
                        const int y = (vv / E.nx) % E.ny;
                        const int z = vv / (E.nx * E.ny);
                        const double* q = E.sc + (int64_t)s * E.L;
                        b[u] *= __ldg(q + x) * __ldg(q + E.nx + y) * __ldg(q + E.nx + E.ny + z);
                    }
                }
            }
        }
        if (!(mask_ok && ((got >> s) & 1ull))) {
            const int i = dep_index(tf, n_sub, 3, s);   // last swept axis of substrate s
            if (i >= 0) wait_count(Q, Q.done + i, (unsigned)(tf[i + 1] - tf[i]) + Q.extra_need, lane);
            if (mask_ok) got |= 1ull << s;
        }
        if (shell) {
            const int64_t lo = (int64_t)k * kEpiChunk;
            const int64_t hi = min(per, lo + kEpiChunk);
            for (int64_t t0 = lo + lane; t0 < hi; t0 += 32 * kEpiUnroll) {
#pragma unroll
                for (int u = 0; u < kEpiUnroll; ++u) {
                    const int64_t t = t0 + 32 * u;
                    if (t < hi) shell_voxel(E, s, bcv[s], t);
                }
            }
            fence_acq_rel_gpu();
            __syncwarp();
            if (lane == 0) atomicAdd(Q.shell_done + s, 1u);
            continue;
        }
        const unsigned need_sh = (dir ? (unsigned)sh_chunks : 0u) + (unsigned)nch;
        if (need_sh > 0 && !(mask_ok && ((got >> (32 + s)) & 1ull))) {
            wait_count(Q, Q.shell_done + s, need_sh + Q.extra_need, lane);
            if (mask_ok) got |= 1ull << (32 + s);
        }
        // entries are distinct voxel-substrate pairs, so no two touch one
        // field element: all gathers first, then the updates
        T f[R];
#pragma unroll
        for (int u = 0; u < R; ++u)
            if (o[u] >= 0) f[u] = E.field[o[u]];
#pragma unroll
        for (int u = 0; u < R; ++u)
            if (o[u] >= 0) E.field[o[u]] = (T)fma(a[u], (double)f[u], b[u]);
    }
}

__device__ __forceinline__ void pair_sync(int bar_id)
{
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
}

// What a pair's two warps share besides the column buffer.
template <typename T>
struct PairShared {
    const int* bck;        // shared copy of the substrates' boundary kinds
    const double* bcv;     // and Dirichlet values
    T* field;              // the field (read and written in place)
    CoefTabs<T> K;         // shared coefficient tables
    int64_t* rbF;          // [32] row bases of F's task (x tasks)
    int64_t* rbB;          // [32] line bases of B's task (-1: padding), written by F
    int* hs;               // [32] substrate of each lane's line in B's task, written by F
    T* handover;           // [32] chain values of the task handed to B
    volatile int* ho;      // task handed over, next task, paired (0/1)
    T* W;                  // column buffer
    int ns, lane, bar_id;
};

// Group count of an axis' lines
template <typename T>
__device__ __forceinline__ int axis_groups(const SweepArgs<T>* sA, int a)
{
    constexpr int G = Groups<T>::G;
    return (sA[a].n + G - 1) / G;
}

// Pair-barrier meetings of a phase in which F eliminates a task of axis
// a_f while B back-substitutes one of axis a_b: B meets once per group of
// its task; F copies group j after meeting j and eliminates it LG meetings
// later.
template <typename T>
__device__ __forceinline__ int phase_iters(const SweepArgs<T>* sA, int a_f, int a_b)
{
    constexpr int LG = Groups<T>::PAIR_LAG;
    return max(axis_groups(sA, a_f) + LG, axis_groups(sA, a_b));
}

// State of a pair's F warp between tasks
struct FState {
    int t;        // task whose forward elimination is due (n_tasks: none)
    int tn;       // the task claimed after it (n_tasks: none)
    int k;        // index of t among this pair's tasks (slot parity k & 1)
    bool solo;    // on its own (first task, or B finished its task alone)
    int iters;    // pair-barrier meetings when not solo
    bool have_line;   // `pre` holds the lines of task t (issued during the previous task)
    LinePre pre;
    unsigned long long acq;  // bit (a - 1) n_sub + s: this warp has acquired the completion of (a - 1, s)
};

__device__ __forceinline__ void mark_acquired(FState& f, int i)
{
    if (i < 64) f.acq |= 1ull << i;
}

// F warp: the forward eliminations of consecutive tasks on axis AXIS, each
// followed by the hand-over to B.  Tasks are claimed in increasing order, so
// a warp's axis never goes back and the three axes run as three loops with
// their own specialised code.  F works one task ahead in its claims: while
// it eliminates task t it already holds the next task tn, and at the start
// it issues the claim of the task after tn and a relaxed read of tn's
// dependency count, so neither round trip is on the pair's path at the
// hand-over (an acquire fence there completes the acquire pattern; only when
// the early read was short does F read the count again).
template <typename T, int AXIS, int MODE, bool NODES>
__device__ __forceinline__ void f_axis(FState& f, const SweepArgs<T>& A, const LineSet& S,
                                       const int64_t* fs, const SweepArgs<T>* sA,
                                       const StepSched& Q, const int* tf, const PairShared<T>& P)
{
    const int NT = Q.n_tasks;
    while (f.t < NT) {
        const TaskRef r = decode_task(tf, Q.n_sub, f.t);
        if (r.a != AXIS) return;
        const Line L = finish_line<MODE, NODES>(
            f.have_line ? f.pre
                        : issue_line<T, AXIS, MODE, NODES>(A, S, fs, P.bck, P.bcv, r, P.lane));
        f.have_line = false;
        const bool has_next = f.tn < NT;
        TaskRef rn{0, 0, 0};
        unsigned need = 0, seen = 0, raw2 = 0;
        int dep = -1;              // completion counter tn waits on (-1: none or acquired)
        if (has_next) {
            rn = decode_task(tf, Q.n_sub, f.tn);
            dep = dep_index(tf, Q.n_sub, rn.a, rn.s);
            if (dep >= 0 && dep < 64 && ((f.acq >> dep) & 1ull)) dep = -1;
            if (dep >= 0) {
                need = (unsigned)(tf[dep + 1] - tf[dep]) + Q.extra_need;
                if (P.lane == 0) seen = ld_relaxed_u32(Q.done + dep);
            }
            if (P.lane == 0) raw2 = atomicAdd(Q.claim, 1u);
            if (rn.a == AXIS) {
                // the next task's lines: their global reads overlap this task
                f.pre = issue_line<T, AXIS, MODE, NODES>(A, S, fs, P.bck, P.bcv, rn, P.lane);
                f.have_line = true;
            }
        }
        const T prev = f_task<T, AXIS, MODE>(A, L, P.field, P.K, P.W, P.ns, P.lane, P.bar_id,
                                             P.rbF, f.k & 1, f.solo, f.iters);
        bool paired = false;
        if (has_next) {
            if (dep < 0) {
                paired = true;
            } else if (__shfl_sync(0xffffffffu, (int)(seen >= need), 0)) {
                fence_acq_rel_gpu();
                mark_acquired(f, dep);
                paired = true;
            } else if (task_ready(Q, tf, rn, P.lane)) {
                mark_acquired(f, dep);
                paired = true;
            }
        }
        // hand task f.t to B: chain values, line bases, substrates, next task
        P.handover[P.lane] = prev;
        P.rbB[P.lane] = L.valid ? L.base : -1;
        P.hs[P.lane] = L.s;
        if (P.lane == 0) {
            P.ho[0] = f.t;
            P.ho[1] = f.tn;
            P.ho[2] = paired ? 1 : 0;
        }
        pair_sync(P.bar_id);                            // hand-over of task f.t
        if (!has_next) {
            f.t = NT;
            return;
        }
        if (paired) {
            f.solo = false;
            f.iters = phase_iters(sA, rn.a, AXIS);
        } else {
            task_wait(Q, tf, rn, P.lane);
            if (dep >= 0) mark_acquired(f, dep);
            pair_sync(P.bar_id);                        // B has finished f.t on its own
            f.solo = true;
            f.iters = 0;
        }
        const unsigned t2 = __shfl_sync(0xffffffffu, raw2, 0);
        f.t = f.tn;
        f.tn = t2 < (unsigned)NT ? (int)t2 : NT;
        ++f.k;
    }
}

// State of a pair's B warp: the task handed over last
template <typename T>
struct BState {
    int t, t_next;
    bool paired;
    int k;
    T x;
};

// B warp (NODES form): the Dirichlet nodes [i0, i1) on the lines of an x or
// y task take their values after the sweep of AXIS (scales of the axes swept
// so far in state p + 1, the others in state p), one node per lane.  The
// warp barrier orders every lane's stores of the task's lines before them.
template <typename T, int AXIS, int MODE>
__device__ __forceinline__ void patch_task_nodes(const SweepArgs<T>& A, const StepSched& Q,
                                                 T* field, int i0, int i1, int s, int lane)
{
    if (i0 == i1) return;
    __syncwarp();
    for (int i = i0 + lane; i < i1; i += 32) {
        const NodePatch e = Q.node_patch[i];
        double v = e.v;
        if (MODE >= 1) {
            const int64_t row = (int64_t)s * A.L;
            const double* sy = AXIS >= 1 ? A.sc_p1 : A.sc_p;
            v = v * (A.sc_p1[row + A.off_x + e.x] * sy[row + A.off_y + e.y] *
                     A.sc_p[row + A.off_z + e.z]);
        }
        field[e.off] = (T)v;
    }
}

// B warp: back substitutions of consecutive tasks on axis AXIS
template <typename T, int AXIS, int MODE, bool NODES>
__device__ __forceinline__ void b_axis(BState<T>& b, const SweepArgs<T>& A, const LineSet& S,
                                       const int64_t* fs, const SweepArgs<T>* sA,
                                       const StepSched& Q, const int* tf, const PairShared<T>& P)
{
    const int NT = Q.n_tasks;
    while (b.t < NT) {
        const TaskRef r = decode_task(tf, Q.n_sub, b.t);
        if (r.a != AXIS) return;
        const bool more = b.t_next < NT;
        const bool paired = more && b.paired;
        int iters = 0;
        if (paired) {
            const TaskRef rn = decode_task(tf, Q.n_sub, b.t_next);
            iters = phase_iters(sA, rn.a, AXIS);
        }
        const int lane = P.lane;
        // the task's node patches (read now, used after the task's stores)
        int ni0 = 0, ni1 = 0;
        if (NODES && AXIS < 2) {
            ni0 = Q.node_task_first[b.t];
            ni1 = Q.node_task_first[b.t + 1];
        }
        auto rel = [&]() {
            if (NODES && AXIS < 2) patch_task_nodes<T, AXIS, MODE>(A, Q, P.field, ni0, ni1, r.s, lane);
            task_done(Q, r, lane);
        };
        b_task<T, AXIS, MODE>(A, S, fs, P.bck, P.bcv, P.field, P.K, P.W, P.ns, P.lane, P.bar_id,
                              r, P.rbB, P.hs, b.k & 1, b.x, paired, iters, rel);
        if (!more) {
            b.t = NT;
            return;
        }
        if (!b.paired) pair_sync(P.bar_id);             // buffer free for F
        pair_sync(P.bar_id);                            // next hand-over
        b.t = P.ho[0];
        b.t_next = P.ho[1];
        b.paired = P.ho[2] != 0;
        b.x = P.handover[P.lane];
        ++b.k;
    }
}

// Dynamic shared memory, in this order: copies of the 3 axes' SweepArgs and
// LineSets; task_first; the line-set prefixes of the 3 axes; the
// coefficient tables of all substrates and axes (ncoef x n_sub x L: forward
// and backward, and their FP32 low parts); the boundary values (n_sub
// doubles) and kinds (n_sub ints); then per pair: the column buffer
// (n_slots x 32), 4 x 32 row / line bases, 32 chain values, 4 hand-over
// words and 32 substrates.  n_slots = G * max over axes of ceil(n / G), so
// the slot schedule of PairSweeper holds for any two axes.  Every part
// starts on a 16-byte boundary.
struct StepSmem {
    size_t args, tf, fs, coef, bc, fixed, pair;
};

__host__ __device__ inline size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename T>
__host__ __device__ inline StepSmem step_smem(int n_sub, int64_t L, int ncoef, int ns)
{
    StepSmem m;
    m.args = round16(3 * sizeof(SweepArgs<T>) + 3 * sizeof(LineSet));
    m.tf = round16(((size_t)3 * n_sub + 1) * sizeof(int));
    m.fs = round16((size_t)3 * (n_sub + 1) * sizeof(int64_t));
    m.coef = round16((size_t)ncoef * n_sub * L * sizeof(T));
    m.bc = round16((size_t)n_sub * (sizeof(double) + sizeof(int)));
    m.fixed = m.args + m.tf + m.fs + m.coef + m.bc;
    m.pair = round16((size_t)ns * 32 * sizeof(T) + 4 * 32 * sizeof(int64_t) + 32 * sizeof(T) +
                     4 * sizeof(int) + 32 * sizeof(int));
    return m;
}

// Coefficient tables the step kernel stages: fa / fb in the rescaled form;
// r / cr in the plain form, with their low parts in FP32.
template <typename T, int MODE>
__host__ __device__ constexpr int step_ncoef()
{
    return (MODE == 0 && sizeof(T) == 4) ? 4 : 2;
}

// The step kernel.  T: element type; MXY: form of the x and y sweeps (0
// plain, 1 rescaled); MZ: form of the z sweep (MXY, or 2: rescaled and
// renormalising); NODES: the context holds Dirichlet nodes (line ends from
// the node end tables, node patches after x and y tasks, node chunks in the
// epilogue; the values before the x sweep are written by a launch ahead).
template <typename T, int MXY, int MZ, bool NODES>
__global__ void __launch_bounds__(64 * Groups<T>::MAX_PAIRS, 1)
    k_step_pair(SweepArgs<T> A0, SweepArgs<T> A1, SweepArgs<T> A2, LineSet S0, LineSet S1,
                LineSet S2, StepSched Q, EpiArgs<T> E, int n_slots)
{
    constexpr int NC = step_ncoef<T, MXY>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int pairs = blockDim.x >> 6;
    const int pair = warp % pairs;
    const bool is_b = warp >= pairs;
    const int n_sub = Q.n_sub;
    const int ns = n_slots;
    const int NT = Q.n_tasks;
    const StepSmem M = step_smem<T>(n_sub, A0.L, NC, ns);

    // the launch arguments of the three axes are read from shared copies:
    // the loop body stores to shared memory, so the compiler reloads them
    // per task instead of keeping all three axes' values live in registers
    SweepArgs<T>* sA = reinterpret_cast<SweepArgs<T>*>(smem_raw);
    LineSet* sS = reinterpret_cast<LineSet*>(smem_raw + 3 * sizeof(SweepArgs<T>));
    int* tf = reinterpret_cast<int*>(smem_raw + M.args);
    int64_t* fs = reinterpret_cast<int64_t*>(smem_raw + M.args + M.tf);  // [3][n_sub+1]
    const int64_t n_coef = (int64_t)n_sub * A0.L;
    T* cf = reinterpret_cast<T*>(smem_raw + M.args + M.tf + M.fs);
    double* bcv = reinterpret_cast<double*>(smem_raw + M.args + M.tf + M.fs + M.coef);
    int* bck = reinterpret_cast<int*>(bcv + n_sub);               // [n_sub]
    unsigned char* pair_area = smem_raw + M.fixed;
    if (threadIdx.x == 0) {
        sA[0] = A0;
        sA[1] = A1;
        sA[2] = A2;
        sS[0] = S0;
        sS[1] = S1;
        sS[2] = S2;
    }
    for (int i = threadIdx.x; i <= 3 * n_sub; i += blockDim.x) tf[i] = Q.task_first[i];
    // the three axes share one table per kind ([s][L], axis offsets within L)
    for (int64_t i = threadIdx.x; i < n_coef; i += blockDim.x) {
        if (MXY >= 1) {
            cf[i] = A0.fa[i];
            cf[n_coef + i] = A0.fb[i];
        } else {
            cf[i] = A0.r[i];
            cf[n_coef + i] = A0.cr[i];
            if (NC == 4) {
                cf[2 * n_coef + i] = A0.r_lo[i];
                cf[3 * n_coef + i] = A0.cr_lo[i];
            }
        }
    }
    for (int i = threadIdx.x; i < n_sub; i += blockDim.x) {
        bcv[i] = A0.bc_value[i];
        bck[i] = A0.bc_kind[i];
    }
    for (int i = threadIdx.x; i <= n_sub; i += blockDim.x) {
        fs[i] = S0.first[i];
        fs[(n_sub + 1) + i] = S1.first[i];
        fs[2 * (n_sub + 1) + i] = S2.first[i];
    }
    __syncthreads();
    const int64_t* fs0 = fs;
    const int64_t* fs1 = fs + (n_sub + 1);
    const int64_t* fs2 = fs + 2 * (n_sub + 1);

    unsigned char* my = pair_area + (size_t)pair * M.pair;
    T* W = reinterpret_cast<T*>(my);
    int64_t* rbF = reinterpret_cast<int64_t*>(my + (size_t)ns * 32 * sizeof(T));
    int64_t* rbB = rbF + 64;
    T* handover = reinterpret_cast<T*>(rbF + 128);
    volatile int* ho = reinterpret_cast<volatile int*>(handover + 32);  // t_cur, t_next, paired
    int* hs = const_cast<int*>(ho) + 4;                                  // [32] substrates
    const int bar_id = 1 + pair;

    PairShared<T> P;
    P.bck = bck;
    P.bcv = bcv;
    P.field = A0.field;
    P.K.a = cf;
    P.K.b = cf + n_coef;
    P.K.a_lo = NC == 4 ? cf + 2 * n_coef : cf;
    P.K.b_lo = NC == 4 ? cf + 3 * n_coef : cf + n_coef;
    P.rbF = rbF;
    P.rbB = rbB;
    P.hs = hs;
    P.handover = handover;
    P.ho = ho;
    P.W = W;
    P.ns = ns;
    P.lane = lane;
    P.bar_id = bar_id;

    if (!is_b) {
        FState f;
        f.t = claim_task(Q, lane);
        f.tn = f.t < NT ? claim_task(Q, lane) : NT;
        f.k = 0;
        f.solo = true;
        f.iters = 0;
        f.have_line = false;
        f.acq = 0ull;
        if (f.t < NT) {
            const TaskRef r0 = decode_task(tf, n_sub, f.t);
            task_wait(Q, tf, r0, lane);
            const int d0 = dep_index(tf, n_sub, r0.a, r0.s);
            if (d0 >= 0) mark_acquired(f, d0);
        } else {
            if (lane == 0) {
                ho[0] = NT;
                ho[1] = NT;
                ho[2] = 0;
            }
            pair_sync(bar_id);                          // nothing for B
        }
        f_axis<T, 0, MXY, NODES>(f, sA[0], sS[0], fs0, sA, Q, tf, P);
        f_axis<T, 1, MXY, NODES>(f, sA[1], sS[1], fs1, sA, Q, tf, P);
        f_axis<T, 2, MZ, NODES>(f, sA[2], sS[2], fs2, sA, Q, tf, P);
    } else {
        BState<T> b;
        pair_sync(bar_id);                              // first hand-over
        b.t = ho[0];
        b.t_next = ho[1];
        b.paired = ho[2] != 0;
        b.x = handover[lane];
        b.k = 0;
        b_axis<T, 0, MXY, NODES>(b, sA[0], sS[0], fs0, sA, Q, tf, P);
        b_axis<T, 1, MXY, NODES>(b, sA[1], sS[1], fs1, sA, Q, tf, P);
        b_axis<T, 2, MZ, NODES>(b, sA[2], sS[2], fs2, sA, Q, tf, P);
    }

    // sweep tasks exhausted for this warp: the step's epilogue
    step_epilogue<T, NODES>(Q, E, tf, bck, bcv, lane);

    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned before = atomicAdd(Q.exit_count, 1u);
        if (before == gridDim.x - 1) {
            // every CTA is past its last claim, wait and completion count
            *Q.claim = 0u;
            for (int i = 0; i < 3 * n_sub; ++i) Q.done[i] = 0u;
            *Q.eclaim = 0u;
            for (int i = 0; i < n_sub; ++i) Q.shell_done[i] = 0u;
            *Q.exit_count = 0u;
            __threadfence();
        }
    }
}

}  // namespace persistent
}  // namespace bfvm
