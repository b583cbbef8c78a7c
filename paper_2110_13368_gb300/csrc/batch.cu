// Batched form: placeholder entry points (filled in by the batched sweep
// implementation).
#include "internal.cuh"

struct bfvm_batch {
    std::string err;
};

extern "C" {

bfvm_status bfvm_batch_create(bfvm_batch** out, bfvm_ctx* const* members, int32_t n_members,
                              void* cuda_stream)
{
    (void)members; (void)n_members; (void)cuda_stream;
    if (out) *out = nullptr;
    return BFVM_ESTATE;
}
bfvm_status bfvm_batch_step(bfvm_batch* b, int32_t n_steps)
{
    (void)b; (void)n_steps;
    return BFVM_ESTATE;
}
bfvm_status bfvm_batch_sync(bfvm_batch* b)
{
    (void)b;
    return BFVM_ESTATE;
}
void bfvm_batch_destroy(bfvm_batch* b) { delete b; }
const char* bfvm_batch_last_error(const bfvm_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
