// The C ABI of include/bfvm.h: argument checks, context state, stream and
// CUDA-graph management.  All numerical work happens in the kernels of
// coeffs.cu, sweeps.cu, sources.cu and adjoint.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include <unordered_map>

#include "internal.cuh"

namespace bfvm {

static thread_local std::string g_create_error;

bfvm_status set_err(Ctx* c, bfvm_status st, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return st;
}

bfvm_status cuda_err(Ctx* c, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
    return set_err(c, e == cudaErrorMemoryAllocation ? BFVM_ENOMEM : BFVM_ECUDA, m);
}

// Device flags, read (and cleared) after the stream is idle: d_err[1] a
// bounded device wait of the one-launch step gave up; d_err[2] a cell
// update (bfvm_update_cells) had invalid cells.
bfvm_status check_wait_flag(Ctx* c)
{
    if (!c->d_err) return BFVM_OK;
    int flag[2] = {0, 0};
    BFVM_CUDA(c, cudaMemcpy(flag, c->d_err + 1, sizeof(flag), cudaMemcpyDeviceToHost));
    if (!flag[0] && !flag[1]) return BFVM_OK;
    BFVM_CUDA(c, cudaMemset(c->d_err + 1, 0, sizeof(flag)));
    if (flag[1])
        return set_err(c, BFVM_EINVAL, "a cell update had invalid cells (positions outside the "
                                       "domain were binned to the nearest voxel); field not valid");
    return set_err(c, BFVM_ETIMEOUT, "a device wait of the step kernel gave up (result not valid)");
}

namespace {

size_t elem_size(const Ctx* c) { return c->precision == 64 ? 8 : 4; }

void drop_graphs(Ctx* c)
{
    if (c->period_graph) cudaGraphExecDestroy(c->period_graph);
    c->period_graph = nullptr;
    c->period_graph_len = 0;
}

void drop_recording(Ctx* c)
{
    for (void* p : c->checkpoints) cudaFree(p);
    c->checkpoints.clear();
    c->recorded = false;
    c->recorded_steps = 0;
}

bool rescaled(const Ctx* c) { return c->precision == 64 && c->variant == 1; }

int period_of(const Ctx* c) { return rescaled(c) ? c->coef.period : 1; }

// Launch `len` steps starting in state 0 as one captured graph.
bfvm_status launch_graph_block(Ctx* c, int len)
{
    if (!c->period_graph || c->period_graph_len != len) {
        drop_graphs(c);
        cudaStream_t cs = nullptr;
        BFVM_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaStream_t saved = c->stream;
        c->stream = cs;
        int64_t launches_before = c->launches;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        bfvm_status st = BFVM_OK;
        if (e == cudaSuccess) {
            int m = period_of(c);
            for (int i = 0; i < len && st == BFVM_OK; ++i) {
                int p = i % m;
                st = launch_step(c, p, rescaled(c) && p == m - 1);
            }
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (st == BFVM_OK && e2 != cudaSuccess) st = cuda_err(c, e2, "cudaStreamEndCapture");
            if (st == BFVM_OK) {
                cudaError_t e3 = cudaGraphInstantiate(&c->period_graph, g, 0);
                if (e3 != cudaSuccess) st = cuda_err(c, e3, "cudaGraphInstantiate");
            }
            if (g) cudaGraphDestroy(g);
        } else {
            st = cuda_err(c, e, "cudaStreamBeginCapture");
        }
        c->stream = saved;
        cudaStreamDestroy(cs);
        c->period_graph_launches = c->launches - launches_before;   // kernels in the graph
        c->launches = launches_before;
        if (st != BFVM_OK) {
            drop_graphs(c);
            return st;
        }
        c->period_graph_len = len;
    }
    BFVM_CUDA(c, cudaGraphLaunch(c->period_graph, c->stream));
    c->launches += c->period_graph_launches;
    return BFVM_OK;
}

bfvm_status check_finite_array(Ctx* c, const double* a, int64_t n, bool nonneg,
                               const char* what)
{
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(a[i]) || (nonneg && a[i] < 0.0))
            return set_err(c, BFVM_EINVAL, std::string(what) + " must be finite" +
                                               (nonneg ? " and >= 0" : ""));
    }
    return BFVM_OK;
}

}  // namespace

bfvm_status copy_in_dense(Ctx* c, const void* src, bool on_device)
{
    size_t es = elem_size(c);
    int64_t rows = (int64_t)c->n_sub * c->nz * c->ny;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->pitch == c->nx)   // rows are contiguous: one linear copy
        BFVM_CUDA(c, cudaMemcpyAsync(c->field, src, es * rows * c->nx, kind, c->stream));
    else
        BFVM_CUDA(c, cudaMemcpy2DAsync(c->field, c->pitch * es, src, c->nx * es, c->nx * es,
                                       rows, kind, c->stream));
    if (!on_device) BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    return BFVM_OK;
}

bfvm_status copy_out_dense(Ctx* c, void* dst, bool on_device)
{
    size_t es = elem_size(c);
    int64_t rows = (int64_t)c->n_sub * c->nz * c->ny;
    const size_t bytes = es * rows * c->nx;
    if (c->scale_state != 0) {
        // the stored field carries a rescale: divide it out while copying
        // (through the context's staging buffer when the target is the host)
        void* tmp = dst;
        if (!on_device) {
            if (c->staging_bytes < bytes) {
                if (c->staging) cudaFree(c->staging);
                c->staging = nullptr;
                c->staging_bytes = 0;
                BFVM_CUDA(c, cudaMalloc(&c->staging, bytes));
                c->staging_bytes = bytes;
            }
            tmp = c->staging;
        }
        bfvm_status st = launch_unscale_copy(c, tmp, c->scale_state);
        if (st == BFVM_OK && !on_device) {
            cudaError_t e = cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) st = cuda_err(c, e, "copy out");
        }
        return st;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->pitch == c->nx)
        BFVM_CUDA(c, cudaMemcpyAsync(dst, c->field, bytes, kind, c->stream));
    else
        BFVM_CUDA(c, cudaMemcpy2DAsync(dst, c->nx * es, c->field, c->pitch * es, c->nx * es,
                                       rows, kind, c->stream));
    if (!on_device) BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    return BFVM_OK;
}

// Store a checkpoint of the current (plain-valued) field, dense FP64.
static bfvm_status push_checkpoint(Ctx* c)
{
    size_t bytes = sizeof(double) * (size_t)c->n_sub * c->nz * c->ny * c->nx;
    void* buf = nullptr;
    BFVM_CUDA(c, cudaMalloc(&buf, bytes));
    c->checkpoints.push_back(buf);
    return launch_unscale_copy(c, buf, c->scale_state);
}

}  // namespace bfvm

using namespace bfvm;

extern "C" {

const char* bfvm_status_string(int32_t s)
{
    switch (s) {
        case BFVM_OK: return "BFVM_OK";
        case BFVM_EINVAL: return "BFVM_EINVAL";
        case BFVM_ENOMEM: return "BFVM_ENOMEM";
        case BFVM_ECUDA: return "BFVM_ECUDA";
        case BFVM_ESTATE: return "BFVM_ESTATE";
        case BFVM_ETIMEOUT: return "BFVM_ETIMEOUT";
        case BFVM_ENONFINITE: return "BFVM_ENONFINITE";
        default: return "BFVM_UNKNOWN";
    }
}

const char* bfvm_last_error(const bfvm_ctx* ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->impl.err.c_str();
}

bfvm_status bfvm_create(bfvm_ctx** out, int32_t nx, int32_t ny, int32_t nz, double dx_um,
                        double dt_min, int32_t n_sub, const double* D, const double* lambda,
                        const int32_t* bc_kind, const double* bc_value, int32_t precision,
                        void* cuda_stream)
{
    if (!out) return set_err(nullptr, BFVM_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return set_err(nullptr, BFVM_EINVAL, "grid edges must be >= 1");
    if (n_sub < 1) return set_err(nullptr, BFVM_EINVAL, "n_sub must be >= 1");
    if (!(dx_um > 0.0) || !isfinite(dx_um)) return set_err(nullptr, BFVM_EINVAL, "dx must be finite and > 0");
    if (!(dt_min > 0.0) || !isfinite(dt_min)) return set_err(nullptr, BFVM_EINVAL, "dt must be finite and > 0");
    if (precision != 64 && precision != 32) return set_err(nullptr, BFVM_EINVAL, "precision must be 64 or 32");
    if (!D || !lambda || !bc_kind || !bc_value) return set_err(nullptr, BFVM_EINVAL, "NULL parameter array");
    int64_t n_vox = (int64_t)nx * ny * nz;
    if (n_vox > (1ll << 33)) return set_err(nullptr, BFVM_EINVAL, "grid too large (limit 2^33 voxels)");
    for (int s = 0; s < n_sub; ++s) {
        if (!isfinite(D[s]) || D[s] < 0.0) return set_err(nullptr, BFVM_EINVAL, "D must be finite and >= 0");
        if (!isfinite(lambda[s]) || lambda[s] < 0.0) return set_err(nullptr, BFVM_EINVAL, "lambda must be finite and >= 0");
        if (bc_kind[s] != BFVM_BC_ZERO_FLUX && bc_kind[s] != BFVM_BC_DIRICHLET)
            return set_err(nullptr, BFVM_EINVAL, "bc_kind must be 0 (zero-flux) or 1 (Dirichlet)");
        if (!isfinite(bc_value[s])) return set_err(nullptr, BFVM_EINVAL, "bc_value must be finite");
    }
    bfvm_ctx* h = new (std::nothrow) bfvm_ctx();
    if (!h) return set_err(nullptr, BFVM_ENOMEM, "host allocation failed");
    Ctx* c = &h->impl;
    c->nx = nx; c->ny = ny; c->nz = nz; c->n_sub = n_sub; c->precision = precision;
    c->dx = dx_um; c->dt = dt_min;
    c->D.assign(D, D + n_sub);
    c->lambda.assign(lambda, lambda + n_sub);
    c->bc_kind.assign(bc_kind, bc_kind + n_sub);
    c->bc_value.assign(bc_value, bc_value + n_sub);
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    c->pitch = ((int64_t)nx + 3) / 4 * 4;
    c->n_field = (int64_t)n_sub * nz * ny * c->pitch;
    c->variant = precision == 64 ? 1 : 0;

    auto fail = [&](bfvm_status st) {
        g_create_error = c->err;
        bfvm_destroy(h);
        return st;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return fail(cuda_err(c, e, "cudaGetDevice"));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, c->device);
    if (e != cudaSuccess) return fail(cuda_err(c, e, "cudaGetDeviceProperties"));
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    size_t es = elem_size(c);
    if ((e = cudaMalloc(&c->field, es * c->n_field)) != cudaSuccess) return fail(cuda_err(c, e, "field"));
    if ((e = cudaMemsetAsync(c->field, 0, es * c->n_field, c->stream)) != cudaSuccess)
        return fail(cuda_err(c, e, "field memset"));
    if ((e = cudaMalloc(&c->d_bc_kind, sizeof(int32_t) * n_sub)) != cudaSuccess) return fail(cuda_err(c, e, "bc"));
    if ((e = cudaMalloc(&c->d_bc_value, sizeof(double) * n_sub)) != cudaSuccess) return fail(cuda_err(c, e, "bc"));
    if ((e = cudaMalloc(&c->d_err, sizeof(int) * 4)) != cudaSuccess) return fail(cuda_err(c, e, "flags"));
    if ((e = cudaMemsetAsync(c->d_err, 0, sizeof(int) * 4, c->stream)) != cudaSuccess)
        return fail(cuda_err(c, e, "flags memset"));
    cudaMemcpyAsync(c->d_bc_kind, bc_kind, sizeof(int32_t) * n_sub, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_bc_value, bc_value, sizeof(double) * n_sub, cudaMemcpyHostToDevice, c->stream);
    bfvm_status st = build_coefficients(c);
    if (st != BFVM_OK) return fail(st);
    if ((st = build_line_tables(c)) != BFVM_OK) return fail(st);
    *out = h;
    return BFVM_OK;
}

void bfvm_destroy(bfvm_ctx* h)
{
    if (!h) return;
    Ctx* c = &h->impl;
    if (c->stream || c->field) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    drop_recording(c);
    for (cudaEvent_t e : c->ev_start) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_stop) cudaEventDestroy(e);
    free_sources(c);
    free_coefficients(c);
    if (c->staging) cudaFree(c->staging);
    c->free_nodes();
    c->free_line_tables();
    if (c->field) cudaFree(c->field);
    if (c->d_bc_kind) cudaFree(c->d_bc_kind);
    if (c->d_bc_value) cudaFree(c->d_bc_value);
    if (c->d_err) cudaFree(c->d_err);
    if (c->slab_tab) cudaFree(c->slab_tab);
    if (c->d_z_starts) cudaFree(c->d_z_starts);
    delete h;
}

bfvm_status bfvm_set_density(bfvm_ctx* h, const void* rho, int32_t on_device)
{
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (!rho) return set_err(c, BFVM_EINVAL, "rho is NULL");
    if (!on_device) {
        // host input: copied into the staging buffer and checked for NaN and
        // Inf there, on the GPU; the field is only replaced when it is clean
        const size_t es = elem_size(c);
        const int64_t n = (int64_t)c->n_sub * c->nz * c->ny * c->nx;
        const size_t bytes = es * n;
        if (c->staging_bytes < bytes) {
            if (c->staging) cudaFree(c->staging);
            c->staging = nullptr;
            c->staging_bytes = 0;
            BFVM_CUDA(c, cudaMalloc(&c->staging, bytes));
            c->staging_bytes = bytes;
        }
        BFVM_CUDA(c, cudaMemcpyAsync(c->staging, rho, bytes, cudaMemcpyHostToDevice, c->stream));
        int bad = 0;
        bfvm_status st = launch_check_finite(c, c->staging, n, &bad);
        if (st != BFVM_OK) return st;
        if (bad) return set_err(c, BFVM_ENONFINITE, "rho holds a NaN or Inf");
        drop_recording(c);
        st = copy_in_dense(c, c->staging, true);
        if (st != BFVM_OK) return st;
        c->scale_state = 0;
        return BFVM_OK;
    }
    drop_recording(c);
    bfvm_status st = copy_in_dense(c, rho, on_device != 0);
    if (st != BFVM_OK) return st;
    c->scale_state = 0;
    return BFVM_OK;
}

bfvm_status bfvm_get_density(bfvm_ctx* h, void* out, int32_t on_device)
{
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (!out) return set_err(c, BFVM_EINVAL, "out is NULL");
    bfvm_status st = copy_out_dense(c, out, on_device != 0);
    if (st != BFVM_OK || on_device) return st;
    return check_wait_flag(c);
}

bfvm_status bfvm_set_cells(bfvm_ctx* h, int64_t n_cells, const double* pos, const double* vol,
                           const double* S, const double* U, const double* rho_star,
                           int32_t on_device)
{
    NvtxRange nvtx("bfvm_set_cells");
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (n_cells < 0) return set_err(c, BFVM_EINVAL, "n_cells must be >= 0");
    drop_recording(c);
    drop_graphs(c);
    if (n_cells == 0) {
        free_sources(c);
        return BFVM_OK;
    }
    if (!pos || !vol || !S || !U || !rho_star) return set_err(c, BFVM_EINVAL, "NULL cell array");
    const int ns = c->n_sub;
    const double* dp = pos;
    const double* dv = vol;
    const double* dS = S;
    const double* dU = U;
    const double* dr = rho_star;
    void* tmp = nullptr;
    if (!on_device) {
        size_t nb = sizeof(double) * (size_t)n_cells * (4 + 3 * ns);
        BFVM_CUDA(c, cudaMalloc(&tmp, nb));
        double* t = static_cast<double*>(tmp);
        double* tp = t;
        double* tv = tp + 3 * n_cells;
        double* tS = tv + n_cells;
        double* tU = tS + n_cells * ns;
        double* tr = tU + n_cells * ns;
        cudaMemcpyAsync(tp, pos, sizeof(double) * 3 * n_cells, cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(tv, vol, sizeof(double) * n_cells, cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(tS, S, sizeof(double) * n_cells * ns, cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(tU, U, sizeof(double) * n_cells * ns, cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(tr, rho_star, sizeof(double) * n_cells * ns, cudaMemcpyHostToDevice, c->stream);
        dp = tp; dv = tv; dS = tS; dU = tU; dr = tr;
    }
    bfvm_status st = build_sources(c, n_cells, dp, dv, dS, dU, dr);
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
    }
    if (st != BFVM_OK) free_sources(c);
    return st;
}

bfvm_status bfvm_step(bfvm_ctx* h, int32_t n_steps)
{
    NvtxRange nvtx("bfvm_step");
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (n_steps < 0) return set_err(c, BFVM_EINVAL, "n_steps must be >= 0");
    if (c->slab >= 0)
        return set_err(c, BFVM_ESTATE, "a z-slab steps with bfvm_slab_forward / "
                                       "bfvm_slab_backward / bfvm_slab_finish");
    if (n_steps == 0) return BFVM_OK;
    const int m = period_of(c);
    bfvm_status st = BFVM_OK;
    if (c->record_every > 0) {
        drop_recording(c);
        for (int t = 0; t < n_steps && st == BFVM_OK; ++t) {
            if (t % c->record_every == 0) st = push_checkpoint(c);
            if (st != BFVM_OK) break;
            int p = c->scale_state;
            st = launch_step(c, p, rescaled(c) && p == m - 1);
            c->scale_state = (p + 1) % m;
            c->steps_taken += 1;
        }
        if (st == BFVM_OK) {
            c->recorded = true;
            c->recorded_steps = n_steps;
        }
        return st;
    }
    int remaining = n_steps;
    const bool graphs = c->use_graphs && !c->time_kernels;
    // graph blocks: a whole rescale period (FP64 rescaled) or 16 steps
    const int block = rescaled(c) ? m : 16;
    while (remaining > 0 && st == BFVM_OK) {
        if (graphs && c->scale_state == 0 && remaining >= block) {
            st = launch_graph_block(c, block);
            remaining -= block;
            c->steps_taken += block;
            continue;
        }
        int p = c->scale_state;
        st = launch_step(c, p, rescaled(c) && p == m - 1);
        c->scale_state = (p + 1) % m;
        remaining -= 1;
        c->steps_taken += 1;
    }
    return st;
}

bfvm_status bfvm_sync(bfvm_ctx* h)
{
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    BFVM_CUDA(c, cudaGetLastError());
    return check_wait_flag(c);
}

bfvm_status bfvm_record(bfvm_ctx* h, int32_t checkpoint_every)
{
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (checkpoint_every < 0) return set_err(c, BFVM_EINVAL, "checkpoint_every must be >= 0");
    if (checkpoint_every > 0 && c->precision != 64)
        return set_err(c, BFVM_EINVAL, "the adjoint needs an FP64 context");
    if (checkpoint_every > 0 && c->slab >= 0)
        return set_err(c, BFVM_ESTATE, "the adjoint covers whole-grid contexts only");
    if (checkpoint_every > 0) {
        bfvm_status st = sync_source_counts(c);
        if (st != BFVM_OK) return st;
    }
    drop_recording(c);
    c->record_every = checkpoint_every;
    return BFVM_OK;
}

bfvm_status bfvm_backward(bfvm_ctx* h, const double* g_final, int32_t checkpoint_every,
                          double* dD, double* dlambda, double* dS, double* dU, double* g0,
                          int32_t on_device)
{
    NvtxRange nvtx("bfvm_backward");
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (c->precision != 64) return set_err(c, BFVM_EINVAL, "the adjoint needs an FP64 context");
    if (!c->recorded) return set_err(c, BFVM_ESTATE, "no recorded forward run (call bfvm_record first)");
    if (checkpoint_every != 0 && checkpoint_every != c->record_every)
        return set_err(c, BFVM_EINVAL, "checkpoint_every differs from the recorded interval");
    if (!g_final || !dD || !dlambda) return set_err(c, BFVM_EINVAL, "NULL gradient buffer");
    if (c->src.n_cells > 0 && (!dS || !dU)) return set_err(c, BFVM_EINVAL, "NULL dS/dU buffer");
    const int64_t nf = (int64_t)c->n_sub * c->nz * c->ny * c->nx;
    const int64_t nc = c->src.n_cells * c->n_sub;
    if (on_device)
        return run_backward(c, g_final, dD, dlambda, dS, dU, g0);
    // host buffers: stage through device memory
    double *dg = nullptr, *dout = nullptr;
    size_t n_out = 2 * c->n_sub + 2 * nc + (g0 ? nf : 0);
    BFVM_CUDA(c, cudaMalloc(&dg, sizeof(double) * nf));
    BFVM_CUDA(c, cudaMalloc(&dout, sizeof(double) * (n_out > 0 ? n_out : 1)));
    BFVM_CUDA(c, cudaMemcpyAsync(dg, g_final, sizeof(double) * nf, cudaMemcpyHostToDevice, c->stream));
    double* o_dD = dout;
    double* o_dl = o_dD + c->n_sub;
    double* o_dS = o_dl + c->n_sub;
    double* o_dU = o_dS + nc;
    double* o_g0 = g0 ? o_dU + nc : nullptr;
    bfvm_status st = run_backward(c, dg, o_dD, o_dl, o_dS, o_dU, o_g0);
    if (st == BFVM_OK) {
        cudaMemcpyAsync(dD, o_dD, sizeof(double) * c->n_sub, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(dlambda, o_dl, sizeof(double) * c->n_sub, cudaMemcpyDeviceToHost, c->stream);
        if (nc > 0) {
            cudaMemcpyAsync(dS, o_dS, sizeof(double) * nc, cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(dU, o_dU, sizeof(double) * nc, cudaMemcpyDeviceToHost, c->stream);
        }
        if (g0) cudaMemcpyAsync(g0, o_g0, sizeof(double) * nf, cudaMemcpyDeviceToHost, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_err(c, e, "backward copy-out");
    }
    cudaFree(dg);
    cudaFree(dout);
    return st;
}

bfvm_status bfvm_kernel_times(bfvm_ctx* h, double* ms, int64_t* counts, int32_t reset)
{
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < c->ev_stop.size(); ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, c->ev_start[i], c->ev_stop[i]);
        int k = c->ev_kind[i];
        c->kt_ms[k] += t;
        c->kt_n[k] += 1;
    }
    for (cudaEvent_t e : c->ev_start) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_stop) cudaEventDestroy(e);
    c->ev_start.clear();
    c->ev_stop.clear();
    c->ev_kind.clear();
    for (int k = 0; k < 5; ++k) {
        if (ms) ms[k] = c->kt_ms[k];
        if (counts) counts[k] = c->kt_n[k];
        if (reset) {
            c->kt_ms[k] = 0.0;
            c->kt_n[k] = 0;
        }
    }
    return BFVM_OK;
}

bfvm_status bfvm_update_cells(bfvm_ctx* h, int64_t n_cells, const double* pos,
                              const double* vol, const double* S, const double* U,
                              const double* rho_star)
{
    NvtxRange nvtx("bfvm_update_cells");
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (c->src.cap == 0) return set_err(c, BFVM_ESTATE, "no cells to update (bfvm_set_cells first)");
    if (n_cells != c->src.cap)
        return set_err(c, BFVM_EINVAL, "bfvm_update_cells keeps the cell count of the last bfvm_set_cells");
    if (!pos || !vol || !S || !U || !rho_star) return set_err(c, BFVM_EINVAL, "NULL cell array");
    if (c->record_every != 0)
        return set_err(c, BFVM_ESTATE, "cells cannot move while a forward run is recorded for the adjoint");
    // graphs captured with host-side entry counts would keep stale grids
    if (c->src.counts_on_host) drop_graphs(c);
    return update_sources(c, pos, vol, S, U, rho_star);
}

bfvm_status bfvm_set_dirichlet_nodes(bfvm_ctx* h, int64_t n_nodes, const int64_t* voxel,
                                     const int32_t* substrate, const double* value,
                                     int32_t on_device)
{
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (n_nodes < 0) return set_err(c, BFVM_EINVAL, "n_nodes must be >= 0");
    if (n_nodes > 0 && (!voxel || !substrate || !value)) return set_err(c, BFVM_EINVAL, "NULL node array");
    if (n_nodes > 0 && c->slab >= 0)
        return set_err(c, BFVM_ESTATE, "Dirichlet nodes are defined for whole-grid contexts");
    if (n_nodes > 0 && c->dims != 3)
        return set_err(c, BFVM_EINVAL, "Dirichlet nodes are defined for the 3-D step");
    std::vector<int64_t> hv(n_nodes);
    std::vector<int32_t> hs(n_nodes);
    std::vector<double> hval(n_nodes);
    if (n_nodes > 0) {
        cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        if (on_device) BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
        BFVM_CUDA(c, cudaMemcpy(hv.data(), voxel, sizeof(int64_t) * n_nodes, k));
        BFVM_CUDA(c, cudaMemcpy(hs.data(), substrate, sizeof(int32_t) * n_nodes, k));
        BFVM_CUDA(c, cudaMemcpy(hval.data(), value, sizeof(double) * n_nodes, k));
    }
    const int64_t n_vox = (int64_t)c->nx * c->ny * c->nz;
    for (int64_t i = 0; i < n_nodes; ++i) {
        if (hv[i] < 0 || hv[i] >= n_vox) return set_err(c, BFVM_EINVAL, "node voxel out of range");
        if (hs[i] < 0 || hs[i] >= c->n_sub) return set_err(c, BFVM_EINVAL, "node substrate out of range");
        if (!isfinite(hval[i])) return set_err(c, BFVM_EINVAL, "node value must be finite");
    }
    // one node per (voxel, substrate): the later one holds
    std::vector<int64_t> key_order;
    std::unordered_map<int64_t, size_t> slot;
    std::vector<int64_t> off;
    std::vector<int32_t> vox32, sub32;
    std::vector<double> val;
    for (int64_t i = 0; i < n_nodes; ++i) {
        const int64_t key = (int64_t)hs[i] * n_vox + hv[i];
        auto it = slot.find(key);
        if (it != slot.end()) {
            val[it->second] = hval[i];
            continue;
        }
        slot.emplace(key, val.size());
        const int64_t v = hv[i];
        const int x = (int)(v % c->nx), y = (int)((v / c->nx) % c->ny), z = (int)(v / ((int64_t)c->nx * c->ny));
        off.push_back((((int64_t)hs[i] * c->nz + z) * c->ny + y) * c->pitch + x);
        vox32.push_back((int32_t)v);
        sub32.push_back(hs[i]);
        val.push_back(hval[i]);
    }
    drop_recording(c);
    drop_graphs(c);
    BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->free_nodes();
    const int64_t m = (int64_t)val.size();
    if (m == 0) return BFVM_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_node_off, sizeof(int64_t) * m)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_node_vox, sizeof(int32_t) * m)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_node_sub, sizeof(int32_t) * m)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_node_val, sizeof(double) * m)) != cudaSuccess) {
        c->free_nodes();
        return cuda_err(c, e, "node tables");
    }
    BFVM_CUDA(c, cudaMemcpy(c->d_node_off, off.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice));
    BFVM_CUDA(c, cudaMemcpy(c->d_node_vox, vox32.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice));
    BFVM_CUDA(c, cudaMemcpy(c->d_node_sub, sub32.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice));
    BFVM_CUDA(c, cudaMemcpy(c->d_node_val, val.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
    c->n_nodes = m;
    std::vector<int64_t> vox64(vox32.begin(), vox32.end());
    const bfvm_status st = build_node_tables(c, vox64, sub32, val, off);
    if (st != BFVM_OK) c->free_nodes();
    return st;
}

bfvm_status bfvm_get_info(const bfvm_ctx* h, int64_t* info)
{
    if (!h || !info) return BFVM_EINVAL;
    const Ctx* c = &h->impl;
    for (int i = 0; i < 16; ++i) info[i] = 0;
    info[0] = c->precision;
    info[1] = c->nx; info[2] = c->ny; info[3] = c->nz; info[4] = c->n_sub;
    info[5] = c->pitch;
    sync_source_counts(const_cast<Ctx*>(c));
    info[6] = c->src.n_seg;
    info[7] = c->steps_taken;
    info[8] = (c->precision == 64) ? c->variant : 0;
    info[9] = c->coef.period;
    info[10] = c->launches;
    info[11] = c->recorded ? c->recorded_steps : 0;
    info[12] = c->dims;
    return BFVM_OK;
}

bfvm_status bfvm_set_option(bfvm_ctx* h, int32_t key, int64_t value)
{
    if (!h) return BFVM_EINVAL;
    Ctx* c = &h->impl;
    if (c->slab >= 0 && (key == 1 || key == 2 || key == 8 || key == 10))
        return set_err(c, BFVM_ESTATE, "a z-slab runs the plain 3-D form with its own z sweep");
    switch (key) {
        case 1:
            if (value != 0 && value != 1) return set_err(c, BFVM_EINVAL, "variant must be 0 or 1");
            if (value == 1 && c->precision != 64)
                return set_err(c, BFVM_EINVAL, "the rescaled sweep is FP64 only");
            if (value == 1 && c->dims != 3)
                return set_err(c, BFVM_EINVAL, "the rescaled sweep renormalises in the z sweep: 3-D only");
            if (c->scale_state != 0) return set_err(c, BFVM_ESTATE, "field is mid-rescale; step to a period end first");
            c->variant = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 2: {
            if (value < 0 || value > 64) return set_err(c, BFVM_EINVAL, "period must be 0..64");
            if (c->scale_state != 0) return set_err(c, BFVM_ESTATE, "field is mid-rescale");
            c->period_override = (int)value;
            drop_graphs(c);
            return build_coefficients(c);
        }
        case 3:
            if (value != 0 && value != 1) return set_err(c, BFVM_EINVAL, "fuse must be 0 or 1");
            c->fuse_sources = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 4:
            if (value != 0 && value != 1) return set_err(c, BFVM_EINVAL, "graphs must be 0 or 1");
            c->use_graphs = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 5:
            if (value != 0 && value != 1) return set_err(c, BFVM_EINVAL, "timing must be 0 or 1");
            c->time_kernels = (int)value;
            return BFVM_OK;
        case 6:
            if (value < 0 || value > 1000000) return set_err(c, BFVM_EINVAL, "grid limit must be >= 0");
            c->grid_limit = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 7:
            if (value != 0 && value != 1) return set_err(c, BFVM_EINVAL, "sweep kernel must be 0 or 1");
            c->sweep_kernel = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 8:
            if (value < 0 || value > 2) return set_err(c, BFVM_EINVAL, "fused step must be 0, 1 or 2");
            c->fused_step = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 9:
            if (value < 0 || value > 1000000) return set_err(c, BFVM_EINVAL, "poll limit must be 0..1e6");
            c->wait_test_polls = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 11:
            if (value < 0 || value > 2) return set_err(c, BFVM_EINVAL, "split solve must be 0, 1 or 2");
            c->split = (int)value;
            drop_graphs(c);
            return BFVM_OK;
        case 10: {
            if (value != 2 && value != 3) return set_err(c, BFVM_EINVAL, "dims must be 2 or 3");
            if (value == c->dims) return BFVM_OK;
            if (value == 2 && c->nz != 1) return set_err(c, BFVM_EINVAL, "the 2-D variant needs nz == 1");
            if (value == 2 && c->n_nodes > 0)
                return set_err(c, BFVM_ESTATE, "Dirichlet nodes are defined for the 3-D step");
            if (c->scale_state != 0) return set_err(c, BFVM_ESTATE, "field is mid-rescale; step to a period end first");
            if (c->record_every != 0)
                return set_err(c, BFVM_ESTATE, "recording for the adjoint: stop it (bfvm_record(0)) before changing dims");
            c->dims = (int)value;
            // the rescaled form renormalises in the z sweep: 2-D runs the plain form
            c->variant = (c->precision == 64 && c->dims == 3) ? 1 : 0;
            drop_graphs(c);
            c->free_line_tables();
            bfvm_status st = build_coefficients(c);
            if (st != BFVM_OK) return st;
            return build_line_tables(c);
        }
        default:
            return set_err(c, BFVM_EINVAL, "unknown option key");
    }
}

}  // extern "C"
