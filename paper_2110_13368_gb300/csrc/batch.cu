// C ABI of the batched form: many independent contexts of uneven sizes
// advanced together, one launch per sweep phase over a flat list of
// (member, 32-line block) tasks (kernels in sweeps.cu), a whole rescale
// period captured as one CUDA graph.
#include <algorithm>
#include <string>

#include "internal.cuh"

struct bfvm_batch {
    bfvm::BatchImpl impl;
};

using namespace bfvm;

namespace {

bfvm_status berr(BatchImpl* b, bfvm_status st, const std::string& msg)
{
    if (b) b->err = msg;
    return st;
}

bfvm_status bcuda(BatchImpl* b, cudaError_t e, const char* what)
{
    return berr(b, e == cudaErrorMemoryAllocation ? BFVM_ENOMEM : BFVM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

bfvm_status launch_block(BatchImpl* b, int len)
{
    if (!b->graph || b->graph_len != len) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        cudaStream_t cs = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamCreate");
        cudaStream_t saved = b->stream;
        b->stream = cs;
        int64_t saved_launches = b->launches;
        bfvm_status st = BFVM_OK;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = bcuda(b, e, "cudaStreamBeginCapture");
        if (st == BFVM_OK) {
            for (int i = 0; i < len && st == BFVM_OK; ++i) {
                int p = i % b->period;
                st = batch_launch_step(b, p, b->rescaled && p == b->period - 1);
            }
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (st == BFVM_OK && e2 != cudaSuccess) st = bcuda(b, e2, "cudaStreamEndCapture");
            if (st == BFVM_OK) {
                e2 = cudaGraphInstantiate(&b->graph, g, 0);
                if (e2 != cudaSuccess) st = bcuda(b, e2, "cudaGraphInstantiate");
            }
            if (g) cudaGraphDestroy(g);
        }
        b->stream = saved;
        cudaStreamDestroy(cs);
        b->launches = saved_launches;
        if (st != BFVM_OK) return berr(b, st, b->err.empty() ? "batched graph capture failed" : b->err);
        b->graph_len = len;
    }
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
    const int per_step = (b->one_launch && b->one_launch_ok) ? 1 : 3 + (b->n_entries > 0 ? 1 : 0);
    b->launches += (int64_t)len * per_step;
    return BFVM_OK;
}

}  // namespace

extern "C" {

bfvm_status bfvm_batch_create(bfvm_batch** out, bfvm_ctx* const* members, int32_t n_members,
                              void* cuda_stream)
{
    if (!out) return BFVM_EINVAL;
    *out = nullptr;
    if (!members || n_members < 1) return BFVM_EINVAL;
    bfvm_batch* h = new (std::nothrow) bfvm_batch();
    if (!h) return BFVM_ENOMEM;
    BatchImpl* b = &h->impl;
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    int period = 64;
    bool all_rescaled = true;
    for (int i = 0; i < n_members; ++i) {
        if (!members[i]) {
            delete h;
            return BFVM_EINVAL;
        }
        Ctx* c = &members[i]->impl;
        if (sync_source_counts(c) != BFVM_OK) {
            delete h;
            return BFVM_ECUDA;
        }
        if (i == 0) b->precision = c->precision;
        if (c->precision != b->precision || c->scale_state != 0 || c->record_every != 0 ||
            c->n_nodes > 0 || c->slab >= 0) {
            delete h;
            return BFVM_ESTATE;
        }
        all_rescaled = all_rescaled && c->precision == 64 && c->variant == 1;
        if (c->coef.period > 0) period = std::min(period, c->coef.period);
        b->members.push_back(c);
    }
    b->rescaled = all_rescaled;
    b->period = b->rescaled ? std::max(period, 1) : 1;
    bfvm_status st = batch_build(b);
    if (st != BFVM_OK) {
        batch_free(b);
        delete h;
        return st;
    }
    *out = h;
    return BFVM_OK;
}

bfvm_status bfvm_batch_step(bfvm_batch* h, int32_t n_steps)
{
    NvtxRange nvtx("bfvm_batch_step");
    if (!h) return BFVM_EINVAL;
    BatchImpl* b = &h->impl;
    if (n_steps < 0) return berr(b, BFVM_EINVAL, "n_steps must be >= 0");
    int remaining = n_steps;
    const int block = b->rescaled ? b->period : 16;
    bfvm_status st = BFVM_OK;
    while (remaining > 0 && st == BFVM_OK) {
        if (b->p == 0 && remaining >= block) {
            st = launch_block(b, block);
            remaining -= block;
            continue;
        }
        st = batch_launch_step(b, b->p, b->rescaled && b->p == b->period - 1);
        if (st != BFVM_OK) st = berr(b, st, "batched step launch failed");
        b->p = b->rescaled ? (b->p + 1) % b->period : 0;
        remaining -= 1;
    }
    for (Ctx* c : b->members) {
        c->scale_state = b->p;
        c->steps_taken += n_steps - remaining;
    }
    return st;
}

bfvm_status bfvm_batch_sync(bfvm_batch* h)
{
    if (!h) return BFVM_EINVAL;
    BatchImpl* b = &h->impl;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(b, e, "batch sync");
    if (b->d_err) {
        int flag = 0;
        e = cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bcuda(b, e, "batch sync");
        if (flag) {
            cudaMemset(b->d_err, 0, sizeof(int));
            return berr(b, BFVM_ETIMEOUT,
                        "a device wait of the batched step gave up (result not valid)");
        }
    }
    return BFVM_OK;
}

bfvm_status bfvm_batch_set_option(bfvm_batch* h, int32_t key, int64_t value)
{
    if (!h) return BFVM_EINVAL;
    BatchImpl* b = &h->impl;
    switch (key) {
        case 1:
            if (value != 0 && value != 1) return berr(b, BFVM_EINVAL, "one-launch mode must be 0 or 1");
            if (value == 1 && !b->one_launch_ok)
                return berr(b, BFVM_EINVAL, "the one-launch step does not fit this batch");
            b->one_launch = value == 1;
            break;
        case 2:
            if (value < 0 || value > 1000000) return berr(b, BFVM_EINVAL, "poll limit must be 0..1e6");
            b->wait_test_polls = (int)value;
            break;
        default:
            return berr(b, BFVM_EINVAL, "unknown batch option key");
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_len = 0;
    return BFVM_OK;
}

void bfvm_batch_destroy(bfvm_batch* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->impl.stream);
    batch_free(&h->impl);
    delete h;
}

const char* bfvm_batch_last_error(const bfvm_batch* h) { return h ? h->impl.err.c_str() : ""; }

bfvm_status bfvm_batch_shape(const bfvm_batch* h, int32_t axis, int32_t* algo, int32_t* warps,
                             double* ms)
{
    if (!h || axis < 0 || axis > 2) return BFVM_EINVAL;
    const BatchImpl* b = &h->impl;
    if (algo) *algo = b->algo[axis];
    if (warps) *warps = b->warps[axis];
    if (ms) {
        ms[0] = b->tune_ms[axis][0];
        ms[1] = b->tune_ms[axis][1];
    }
    return BFVM_OK;
}

bfvm_status bfvm_batch_set_shape(bfvm_batch* h, int32_t axis, int32_t algo, int32_t warps)
{
    if (!h) return BFVM_EINVAL;
    BatchImpl* b = &h->impl;
    bfvm_status st = batch_set_shape(b, axis, algo, warps);
    if (st != BFVM_OK)
        return berr(b, st, "unsupported line-block shape (PCR: x lines of at most 128 voxels; "
                           "Thomas: as many warps as the line buffers fit)");
    return BFVM_OK;
}

bfvm_status bfvm_batch_info(const bfvm_batch* h, int64_t* info)
{
    if (!h || !info) return BFVM_EINVAL;
    const BatchImpl* b = &h->impl;
    for (int i = 0; i < 8; ++i) info[i] = 0;
    info[0] = (int64_t)b->members.size();
    info[1] = b->precision;
    info[2] = b->rescaled ? 1 : 0;
    info[3] = b->period;
    info[4] = b->n_tasks[0] + b->n_tasks[1] + b->n_tasks[2];
    info[5] = b->n_entries;
    info[6] = b->launches;
    info[7] = b->p;
    return BFVM_OK;
}

}  // extern "C"
