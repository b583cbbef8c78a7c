// The batched form's step as one persistent launch (included by sweeps.cu
// after sweep_step.cuh, whose scheduler, warp pairs and epilogue pieces it
// reuses over a task list that spans many members).
//
// Tasks: (axis a, group g, block j), where a group is one substrate of one
// member (NS groups in all, a member's groups consecutive) and a block is
// 32 lines of the group's line set on axis a.  They are numbered
// axis-major: every member's x tasks, then every member's y tasks, then the
// z tasks, so the dependency of a task (the previous axis of its own group)
// lies about a third of the list earlier.  task_first[a NS + g] is the first
// task of (a, g) and done[a NS + g] counts its completed tasks: StepSched
// and its waits are the single-context ones with n_sub replaced by NS.
//
// A task's member arguments (its axis' SweepArgs in the launch's rescale
// state) are copied into a shared slot of the pair one task ahead: F issues
// the reads of task k + 1's arguments (k = the pair's task count) before it
// eliminates task k and stores them after; B reads the slot of the task it
// back-substitutes.  Three slots rotate, so F never writes the slot B is
// reading.  The task's coefficient rows are staged the same way: F copies
// them (cp.async, with the task's first column copies) into one of three
// rotating shared slots, where both warps read them as broadcasts.  A
// group's line set is one entry of the group table.
//
// Epilogue: the Dirichlet shell and the cell sources of every group, in
// chunks claimed after the sweep tasks, each waiting on the last swept axis
// of its group (the sources also on the group's shell), as in the
// single-context step.
#pragma once

namespace bfvm {
namespace persistent {

// One (axis, group) of the task list.
struct BGroup {
    int m;          // member
    int s;          // substrate within the member
    int lo_a, cnt_a, lo_b;   // line set: first value and count of the fast other
                             // coordinate, first value of the slow one
    int n;          // line length (extent of the axis)
    int dir;        // Dirichlet substrate
    int pad;
    int64_t n_lines;
    double v;       // Dirichlet value
};

// One member: the three axes' sweep arguments of the launch's rescale
// state, and its epilogue arguments.
template <typename T>
struct BMember {
    SweepArgs<T> A[3];
    EpiArgs<T> E;
    int n_sub;
    int g0;         // its first group
};

template <typename T>
__host__ __device__ constexpr int args_words()
{
    return (int)((sizeof(SweepArgs<T>) + 7) / 8);
}
static_assert(sizeof(SweepArgs<double>) % 8 == 0 && args_words<double>() <= 32 &&
                  args_words<float>() <= 32,
              "a warp copies a member's sweep arguments one 8-byte word per lane");

// Task number -> (axis, group, block): the last (a, g) entry of task_first
// that starts at or before t (entries of empty groups share their start
// with the next one, so the last such entry is the one holding t).
__device__ __forceinline__ TaskRef decode_task_b(const int* tf, int ns, int t)
{
    int lo = 0, hi = 3 * ns;   // tf[lo] <= t < tf[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tf[mid] <= t) lo = mid;
        else hi = mid;
    }
    TaskRef r;
    r.a = lo / ns;
    r.s = lo - r.a * ns;
    r.j = t - tf[lo];
    return r;
}

// The line of this lane in block j of group Gp (padding lanes past the
// group's end repeat its last line and are not stored); the reads of the
// Dirichlet scales are issued here, their arithmetic is finish_line's.
template <typename T, int AXIS, int MODE>
__device__ __forceinline__ LinePre issue_line_b(const SweepArgs<T>& A, const BGroup& Gp, int j,
                                                int lane)
{
    LinePre P;
    int64_t t = (int64_t)j * 32 + lane;
    P.valid = t < Gp.n_lines;
    if (!P.valid) t = Gp.n_lines - 1;
    const int s = Gp.s;
    P.s = s;
    const int a = Gp.lo_a + (int)(t % Gp.cnt_a);
    const int b = Gp.lo_b + (int)(t / Gp.cnt_a);
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
    P.dir = Gp.dir != 0;
    P.v = Gp.v;
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

// What a pair's two warps share in the batched kernel.
template <typename T>
struct BPairShared {
    SweepArgs<T>* slot;    // [3] member arguments of the pair's tasks k mod 3
    int64_t* rbF;
    int64_t* rbB;
    int* hs;
    T* handover;
    double* hinv;          // [32] MODE 2: inverse of the other axes' scales of B's lines
    volatile int* ho;      // task handed over, next task, paired (0/1), pair-barrier
                           // meetings, and the handed task's axis, group, block
    T* W;
    unsigned char* cslot;  // [3] coefficient rows of the pair's tasks k mod 3
    size_t cslot_bytes;
    int ns, lane, bar_id;
};

// Coefficient rows of one task staged in shared memory: the forward and
// backward coefficients (fa / fb of the rescaled form, r / cr of the plain
// form), their FP32 low parts, and (renormalising z sweep) the inverse
// output scales, each indexed by the element k of the line.
template <typename T>
__host__ __device__ constexpr int coef_rows()
{
    return sizeof(T) == 4 ? 4 : 2;
}

template <typename T>
__host__ __device__ inline size_t cslot_size(int n_slots)
{
    return round16((size_t)coef_rows<T>() * n_slots * sizeof(T) + (size_t)n_slots * sizeof(double));
}

template <typename T, int AXIS, int MODE>
__device__ __forceinline__ CoefRow<T> slot_coef_row(const SweepArgs<T>& A, const unsigned char* cs,
                                                    int ns, int s)
{
    const T* t = reinterpret_cast<const T*>(cs);
    CoefRow<T> C;
    C.a = t;
    C.b = t + ns;
    C.a_lo = coef_rows<T>() == 4 ? t + 2 * ns : t;
    C.b_lo = coef_rows<T>() == 4 ? t + 3 * ns : t + ns;
    C.o = reinterpret_cast<const double*>(t + coef_rows<T>() * ns);
    C.c = (T)0;
    C.c_lo = (T)0;
    if (MODE == 0) {
        C.c = A.cvec[s * 3 + AXIS];
        if (sizeof(T) == 4) C.c_lo = A.cvec_lo[s * 3 + AXIS];
    }
    return C;
}

// F: copy (cp.async, in the commit group of the task's first column copies)
// the coefficient rows of substrate s of a task on axis `axis` into slot cs
template <typename T, int MXY, int MZ>
__device__ __forceinline__ void stage_coefs(const SweepArgs<T>& A, int axis, int s,
                                            unsigned char* cs, int ns, int lane)
{
    T* t = reinterpret_cast<T*>(cs);
    const int mode = axis == 2 ? MZ : MXY;
    const int64_t row = (int64_t)s * A.L + A.axis_off;
    const T* a;
    const T* b;
    if (mode >= 1) {
        a = reinterpret_cast<const T*>(A.fa) + row;
        b = reinterpret_cast<const T*>(A.fb) + row;
    } else {
        a = A.r + row;
        b = A.cr + row;
    }
    for (int i = lane; i < A.n; i += 32) {
        cp_async_elem(t + i, a + i);
        cp_async_elem(t + ns + i, b + i);
        if (coef_rows<T>() == 4) {
            cp_async_elem(t + 2 * ns + i, A.r_lo + row + i);
            cp_async_elem(t + 3 * ns + i, A.cr_lo + row + i);
        }
        if (mode == 2) {
            double* o = reinterpret_cast<double*>(t + coef_rows<T>() * ns);
            cp_async_elem(o + i, A.isc_p1 + row + i);
        }
    }
}

struct BFState {
    int t, tn, k;
    int cnext, cend;  // the rest of the pair's claimed chunk
    bool solo;
    int iters;
    TaskRef r;        // decoded t
    LinePre pre;      // lines of t
};

// Copy of task k + 1's member arguments: each lane reads words of the
// table (before the elimination of task k) and stores them to the slot
// (after it).
template <typename T>
struct ArgsCopy {
    uint64_t w;
    __device__ __forceinline__ void load(const BMember<T>* Dm, int m, int a, int lane)
    {
        if (lane < args_words<T>())
            w = __ldg(reinterpret_cast<const unsigned long long*>(&Dm[m].A[a]) + lane);
    }
    __device__ __forceinline__ void store(SweepArgs<T>* dst, int lane) const
    {
        if (lane < args_words<T>()) reinterpret_cast<uint64_t*>(dst)[lane] = w;
    }
};

// Copy-ahead distance of F in the batched kernel, in groups (measured on
// the 256-member workload: FP64 alike with 2 and 3, FP32 6 % faster with the
// pair default than with 2)
template <typename T>
struct BatchLag {
    static constexpr int LG = Groups<T>::PAIR_LAG;
};

// Tasks claimed at a time by a pair: consecutive tasks, mostly of one group,
// so the claims, dependency checks and acquire fences of the later ones are
// skipped.  Measured on the 256-member workload (updates/s for 1, 2, 4, 8):
// FP64 4.31e10, 4.47e10, 4.60e10, 4.65e10; FP32 7.16e10, 6.96e10, 6.51e10,
// 5.62e10 (its shorter tasks end the step less evenly in larger chunks).
template <typename T>
struct BatchChunk {
    static constexpr int C = sizeof(T) == 8 ? 8 : 1;
};

// F: copies and forward elimination of a task with coefficient row C (see
// f_task of the single-context step)
template <typename T, int AXIS, int MODE>
__device__ __forceinline__ T f_task_b(const SweepArgs<T>& A, const Line& L, const CoefRow<T>& C,
                                      T* W, int ns, int lane, int bar_id, int64_t* rbF, int q,
                                      bool solo, int iters)
{
    constexpr int G = Groups<T>::G;
    PairSweeper<T, AXIS, MODE, BatchLag<T>::LG, false> sw{A, W, A.field, A.field, axis_stride(A, AXIS),
                                                   A.n, ns, lane, bar_id};
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

template <typename T>
__device__ __forceinline__ int line_groups(int n)
{
    return (n + Groups<T>::G - 1) / Groups<T>::G;
}

// F warp of the batched kernel: eliminations of consecutive tasks on axis
// AXIS (see f_axis of the single-context step for the hand-over protocol).
// MXY / MZ: forms of the x and y sweeps and of the z sweep.
template <typename T, int AXIS, int MXY, int MZ>
__device__ __forceinline__ void f_axis_b(BFState& f, const BMember<T>* Dm, const BGroup* grp,
                                         const int* tf, const int* gmem, const StepSched& Q,
                                         const BPairShared<T>& P)
{
    constexpr int MODE = AXIS == 2 ? MZ : MXY;
    constexpr int LG = BatchLag<T>::LG;
    const int NT = Q.n_tasks;
    const int NS = Q.n_sub;
    while (f.t < NT) {
        const TaskRef r = f.r;
        if (r.a != AXIS) return;
        const SweepArgs<T>& A = P.slot[f.k % 3];
        const Line L = finish_line<MODE>(f.pre);
        const bool has_next = f.tn < NT;
        TaskRef rn{0, 0, 0};
        unsigned need = 0, seen = 0, raw2 = 0;
        int dep = -1;
        BGroup gn;
        ArgsCopy<T> cp;
        bool same = false;   // tn is in t's group: its dependency is already acquired
        bool from_chunk = false;
        if (has_next) {
            rn = decode_task_b(tf, NS, f.tn);
            same = rn.a == r.a && rn.s == r.s;
            dep = same ? -1 : dep_index(tf, NS, rn.a, rn.s);
            if (dep >= 0) {
                need = (unsigned)(tf[dep + 1] - tf[dep]) + Q.extra_need;
                if (P.lane == 0) seen = ld_relaxed_u32(Q.done + dep);
            }
            from_chunk = f.cnext < f.cend;
            if (!from_chunk && P.lane == 0) raw2 = atomicAdd(Q.claim, (unsigned)BatchChunk<T>::C);
            gn = grp[(int64_t)rn.a * NS + rn.s];
            cp.load(Dm, gmem[rn.s], rn.a, P.lane);
        }
        const CoefRow<T> C =
            slot_coef_row<T, AXIS, MODE>(A, P.cslot + (f.k % 3) * P.cslot_bytes, P.ns, L.s);
        const T prev = f_task_b<T, AXIS, MODE>(A, L, C, P.W, P.ns, P.lane, P.bar_id, P.rbF,
                                               f.k & 1, f.solo, f.iters);
        bool paired = false;
        if (has_next) {
            if (dep < 0) {
                paired = true;
            } else if (__shfl_sync(0xffffffffu, (int)(seen >= need), 0)) {
                fence_acq_rel_gpu();
                paired = true;
            } else if (task_ready(Q, tf, rn, P.lane)) {
                paired = true;
            }
        }
        const int iters = has_next ? max(line_groups<T>(gn.n) + LG, line_groups<T>(A.n)) : 0;
        // hand task f.t to B: chain values, line bases, substrates, next task
        P.handover[P.lane] = prev;
        P.rbB[P.lane] = L.valid ? L.base : -1;
        P.hs[P.lane] = L.s;
        if (MODE == 2) P.hinv[P.lane] = L.inv_other;
        if (P.lane == 0) {
            P.ho[0] = f.t;
            P.ho[1] = f.tn;
            P.ho[2] = paired ? 1 : 0;
            P.ho[3] = iters;
            P.ho[4] = r.a;
            P.ho[5] = r.s;
            P.ho[6] = r.j;
        }
        if (has_next) cp.store(&P.slot[(f.k + 1) % 3], P.lane);
        pair_sync(P.bar_id);                            // hand-over of task f.t
        if (!has_next) {
            f.t = NT;
            return;
        }
        if (paired) {
            f.solo = false;
            f.iters = iters;
        } else {
            task_wait(Q, tf, rn, P.lane);
            pair_sync(P.bar_id);                        // B has finished f.t on its own
            f.solo = true;
            f.iters = 0;
        }
        unsigned t2;
        if (from_chunk) {
            t2 = (unsigned)f.cnext++;
        } else {
            t2 = __shfl_sync(0xffffffffu, raw2, 0);
            f.cnext = (int)min((unsigned)NT, t2 + 1u);
            f.cend = (int)min((unsigned)NT, t2 + (unsigned)BatchChunk<T>::C);
        }
        f.t = f.tn;
        f.tn = t2 < (unsigned)NT ? (int)t2 : NT;
        f.r = rn;
        ++f.k;
        // the next task's lines and coefficient rows, from its argument slot
        // (stored above; the barrier ordered the stores of every lane)
        const SweepArgs<T>& An = P.slot[f.k % 3];
        stage_coefs<T, MXY, MZ>(An, rn.a, gn.s, P.cslot + (f.k % 3) * P.cslot_bytes, P.ns, P.lane);
        if (rn.a == 0) f.pre = issue_line_b<T, 0, MXY>(An, gn, rn.j, P.lane);
        else if (rn.a == 1) f.pre = issue_line_b<T, 1, MXY>(An, gn, rn.j, P.lane);
        else f.pre = issue_line_b<T, 2, MZ>(An, gn, rn.j, P.lane);
    }
}

template <typename T>
struct BBState {
    int t, t_next;
    bool paired;
    int k;
    int iters;
    TaskRef r;    // decoded t (handed over by F)
    T x;
};

// B warp of the batched kernel: back substitutions on axis AXIS
template <typename T, int AXIS, int MODE>
__device__ __forceinline__ void b_axis_b(BBState<T>& b, const int* tf, const StepSched& Q,
                                         const BPairShared<T>& P)
{
    constexpr int G = Groups<T>::G;
    const int NT = Q.n_tasks;
    while (b.t < NT) {
        const TaskRef r = b.r;
        if (r.a != AXIS) return;
        const bool more = b.t_next < NT;
        const bool paired = more && b.paired;
        const int lane = P.lane;
        const SweepArgs<T>& A = P.slot[b.k % 3];
        auto rel = [&]() { task_done(Q, r, lane); };
        {
            PairSweeper<T, AXIS, MODE, BatchLag<T>::LG, false> sw{A, P.W, A.field, A.field,
                                                           axis_stride(A, AXIS), A.n, P.ns,
                                                           lane, P.bar_id};
            Line L;
            const int64_t hb = P.rbB[lane];
            L.valid = hb >= 0;
            L.base = L.valid ? hb : 0;
            L.s = P.hs[lane];
            L.dir = false;
            L.end0 = L.end1 = 0.0;
            L.inv_other = (MODE == 2) ? P.hinv[lane] : 1.0;
            const CoefRow<T> C =
                slot_coef_row<T, AXIS, MODE>(A, P.cslot + (b.k % 3) * P.cslot_bytes, P.ns, L.s);
            int64_t rv[G];
            sw.load_rows(P.rbB, rv);
            if (b.k & 1) sw.template b_block<1>(L, C, b.x, P.rbB, rv, paired, b.iters, rel);
            else sw.template b_block<0>(L, C, b.x, P.rbB, rv, paired, b.iters, rel);
        }
        if (!more) {
            b.t = NT;
            return;
        }
        if (!b.paired) pair_sync(P.bar_id);             // buffer free for F
        pair_sync(P.bar_id);                            // next hand-over
        b.t = P.ho[0];
        b.t_next = P.ho[1];
        b.paired = P.ho[2] != 0;
        b.iters = P.ho[3];
        b.r.a = P.ho[4];
        b.r.s = P.ho[5];
        b.r.j = P.ho[6];
        b.x = P.handover[P.lane];
        ++b.k;
    }
}

// Epilogue of the batched step: for each group (in group order), its shell
// chunks (Dirichlet) once its last swept axis is complete, then its source
// chunks once its shell is complete too.
template <typename T>
__device__ __forceinline__ void step_epilogue_b(const StepSched& Q, const BMember<T>* Dm,
                                                const BGroup* grp, const int64_t* epi_first,
                                                const int* tf, int lane)
{
    const int NS = Q.n_sub;
    for (;;) {
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(Q.eclaim, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= (unsigned)Q.n_epi_chunks) return;
        int lo = 0, hi = NS;   // epi_first[lo] <= c < epi_first[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(epi_first + mid) <= (int64_t)c) lo = mid;
            else hi = mid;
        }
        const int g = lo;
        int k = (int)((int64_t)c - __ldg(epi_first + g));
        const BGroup& Gg = grp[(int64_t)2 * NS + g];
        const int s = Gg.s;
        const EpiArgs<T>& E = Dm[Gg.m].E;
        const int n_sub = Dm[Gg.m].n_sub;
        const int i = dep_index(tf, NS, 3, g);   // last swept axis of the group
        const int sh_chunks = Gg.dir ? (int)epi_shell_chunks_z(E.nx, E.ny, E.nz, E.zf) : 0;
        const bool shell = k < sh_chunks;
        // a source chunk reads its entries before its waits (see
        // step_epilogue of the single-context step)
        constexpr int R = kEpiChunk / 32;
        int64_t o[R];
        double a[R], bb[R];
        if (!shell) {
            const int64_t n_seg = E.d_nseg ? *E.d_nseg : E.n_seg;
            const int64_t lo_g = (int64_t)(k - sh_chunks) * kEpiChunk;
            const int64_t hi_g = min(n_seg, lo_g + kEpiChunk);
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int64_t gg = lo_g + lane + 32 * u;
                o[u] = -1;
                if (gg < hi_g) {
                    const int64_t e = gg * n_sub + s;
                    o[u] = __ldg(E.off + e);
                    a[u] = __ldg(E.alpha + e);
                    bb[u] = __ldg(E.beta + e);
                    if (E.sc) {
                        const int32_t vv = __ldg(E.vox + e);
                        const int x = vv % E.nx;
                        const int y = (vv / E.nx) % E.ny;
                        const int z = vv / (E.nx * E.ny);
                        const double* q = E.sc + (int64_t)s * E.L;
                        bb[u] *= __ldg(q + x) * __ldg(q + E.nx + y) * __ldg(q + E.nx + E.ny + z);
                    }
                }
            }
        }
        if (i >= 0) wait_count(Q, Q.done + i, (unsigned)(tf[i + 1] - tf[i]) + Q.extra_need, lane);
        if (shell) {
            const int64_t per = shell_count_z(E.nx, E.ny, E.nz, E.zf);
            // without z faces the enumeration starts past its z planes
            const int64_t skip = E.zf ? 0 : 2 * (int64_t)E.nx * E.ny;
            const int64_t lo_t = (int64_t)k * kEpiChunk;
            const int64_t hi_t = min(per, lo_t + kEpiChunk);
            for (int64_t t0 = lo_t + lane; t0 < hi_t; t0 += 32 * kEpiUnroll) {
#pragma unroll
                for (int u = 0; u < kEpiUnroll; ++u) {
                    const int64_t t = t0 + 32 * u;
                    if (t < hi_t) shell_voxel(E, s, Gg.v, t + skip);
                }
            }
            fence_acq_rel_gpu();
            __syncwarp();
            if (lane == 0) atomicAdd(Q.shell_done + g, 1u);
            continue;
        }
        if (Gg.dir) wait_count(Q, Q.shell_done + g, (unsigned)sh_chunks + Q.extra_need, lane);
        T f[R];
#pragma unroll
        for (int u = 0; u < R; ++u)
            if (o[u] >= 0) f[u] = E.field[o[u]];
#pragma unroll
        for (int u = 0; u < R; ++u)
            if (o[u] >= 0) E.field[o[u]] = (T)fma(a[u], (double)f[u], bb[u]);
    }
}

// Dynamic shared memory of the batched kernel: task_first [3 NS + 1] and
// the group -> member map [NS] (ints), then per pair: the column buffer
// (n_slots x 32), 4 x 32 row / line bases, 32 chain values, 32 inverse
// scales, 8 hand-over words, 32 substrates, 3 argument slots and 3
// coefficient slots.
struct BatchSmem {
    size_t tab, pair;
};

template <typename T>
__host__ __device__ inline size_t pair_head_bytes(int n_slots)
{
    return round16((size_t)n_slots * 32 * sizeof(T) + 4 * 32 * sizeof(int64_t) + 32 * sizeof(T) +
                   32 * sizeof(double) + 8 * sizeof(int) + 32 * sizeof(int));
}

template <typename T>
__host__ __device__ inline BatchSmem batch_smem(int ns_groups, int n_slots)
{
    BatchSmem m;
    m.tab = round16(((size_t)3 * ns_groups + 1 + ns_groups) * sizeof(int));
    m.pair = pair_head_bytes<T>(n_slots) + round16(3 * sizeof(SweepArgs<T>)) +
             3 * cslot_size<T>(n_slots);
    return m;
}

// The batched step.  T, MXY, MZ as in k_step_pair.  Dm: the member table of
// the launch's rescale state; Q.n_sub is the group count NS.
template <typename T, int MXY, int MZ>
__global__ void __launch_bounds__(64 * Groups<T>::MAX_PAIRS, 1)
    k_batch_step_pair(const BMember<T>* __restrict__ Dm, const BGroup* __restrict__ grp,
                      const int64_t* __restrict__ epi_first, const int* __restrict__ gmem_global,
                      StepSched Q, int n_slots)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int last_cta;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int pairs = blockDim.x >> 6;
    const int pair = warp % pairs;
    const bool is_b = warp >= pairs;
    const int NS = Q.n_sub;
    const int NT = Q.n_tasks;
    const BatchSmem M = batch_smem<T>(NS, n_slots);

    int* tf = reinterpret_cast<int*>(smem_raw);
    int* gmem = tf + 3 * NS + 1;
    for (int i = threadIdx.x; i <= 3 * NS; i += blockDim.x) tf[i] = Q.task_first[i];
    for (int i = threadIdx.x; i < NS; i += blockDim.x) gmem[i] = gmem_global[i];
    __syncthreads();

    unsigned char* my = smem_raw + M.tab + (size_t)pair * M.pair;
    T* W = reinterpret_cast<T*>(my);
    int64_t* rbF = reinterpret_cast<int64_t*>(my + (size_t)n_slots * 32 * sizeof(T));
    int64_t* rbB = rbF + 64;
    T* handover = reinterpret_cast<T*>(rbF + 128);
    double* hinv = reinterpret_cast<double*>(handover + 32);
    volatile int* ho = reinterpret_cast<volatile int*>(hinv + 32);
    int* hs = const_cast<int*>(ho) + 8;
    SweepArgs<T>* slot = reinterpret_cast<SweepArgs<T>*>(my + pair_head_bytes<T>(n_slots));
    unsigned char* cslot = my + pair_head_bytes<T>(n_slots) + round16(3 * sizeof(SweepArgs<T>));

    BPairShared<T> P;
    P.slot = slot;
    P.rbF = rbF;
    P.rbB = rbB;
    P.hs = hs;
    P.handover = handover;
    P.hinv = hinv;
    P.ho = ho;
    P.W = W;
    P.cslot = cslot;
    P.cslot_bytes = cslot_size<T>(n_slots);
    P.ns = n_slots;
    P.lane = lane;
    P.bar_id = 1 + pair;

    if (!is_b) {
        BFState f;
        {
            // the first task and the next one: from the first claimed chunk,
            // or (a chunk of one task) from a second claim
            constexpr unsigned C = (unsigned)BatchChunk<T>::C;
            unsigned c0 = 0;
            if (lane == 0) c0 = atomicAdd(Q.claim, C);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            f.t = c0 < (unsigned)NT ? (int)c0 : NT;
            f.cnext = (int)min((unsigned)NT, c0 + 1u);
            f.cend = (int)min((unsigned)NT, c0 + C);
            if (f.cnext < f.cend) {
                f.tn = f.cnext++;
            } else if (f.t < NT) {
                unsigned c1 = 0;
                if (lane == 0) c1 = atomicAdd(Q.claim, C);
                c1 = __shfl_sync(0xffffffffu, c1, 0);
                f.tn = c1 < (unsigned)NT ? (int)c1 : NT;
                f.cnext = (int)min((unsigned)NT, c1 + 1u);
                f.cend = (int)min((unsigned)NT, c1 + C);
            } else {
                f.tn = NT;
            }
        }
        f.k = 0;
        f.solo = true;
        f.iters = 0;
        if (f.t < NT) {
            f.r = decode_task_b(tf, NS, f.t);
            ArgsCopy<T> cp;
            cp.load(Dm, gmem[f.r.s], f.r.a, lane);
            const BGroup g0 = grp[(int64_t)f.r.a * NS + f.r.s];
            cp.store(&slot[0], lane);
            __syncwarp();
            task_wait(Q, tf, f.r, lane);
            stage_coefs<T, MXY, MZ>(slot[0], f.r.a, g0.s, cslot, n_slots, lane);
            if (f.r.a == 0) f.pre = issue_line_b<T, 0, MXY>(slot[0], g0, f.r.j, lane);
            else if (f.r.a == 1) f.pre = issue_line_b<T, 1, MXY>(slot[0], g0, f.r.j, lane);
            else f.pre = issue_line_b<T, 2, MZ>(slot[0], g0, f.r.j, lane);
        } else {
            if (lane == 0) {
                ho[0] = NT;
                ho[1] = NT;
                ho[2] = 0;
                ho[3] = 0;
                ho[4] = 3;   // no axis: B's loops end at once
            }
            pair_sync(P.bar_id);                        // nothing for B
        }
        f_axis_b<T, 0, MXY, MZ>(f, Dm, grp, tf, gmem, Q, P);
        f_axis_b<T, 1, MXY, MZ>(f, Dm, grp, tf, gmem, Q, P);
        f_axis_b<T, 2, MXY, MZ>(f, Dm, grp, tf, gmem, Q, P);
    } else {
        BBState<T> b;
        pair_sync(P.bar_id);                            // first hand-over
        b.t = ho[0];
        b.t_next = ho[1];
        b.paired = ho[2] != 0;
        b.iters = ho[3];
        b.r.a = ho[4];
        b.r.s = ho[5];
        b.r.j = ho[6];
        b.x = handover[lane];
        b.k = 0;
        b_axis_b<T, 0, MXY>(b, tf, Q, P);
        b_axis_b<T, 1, MXY>(b, tf, Q, P);
        b_axis_b<T, 2, MZ>(b, tf, Q, P);
    }

    step_epilogue_b<T>(Q, Dm, grp, epi_first, tf, lane);

    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_cta = atomicAdd(Q.exit_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last_cta) {
        // every CTA is past its last claim, wait and completion count
        for (int i = threadIdx.x; i < 3 * NS; i += blockDim.x) Q.done[i] = 0u;
        for (int i = threadIdx.x; i < NS; i += blockDim.x) Q.shell_done[i] = 0u;
        if (threadIdx.x == 0) {
            *Q.claim = 0u;
            *Q.eclaim = 0u;
            *Q.exit_count = 0u;
        }
        __threadfence();
    }
}

}  // namespace persistent
}  // namespace bfvm
