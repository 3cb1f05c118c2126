// osmodi_solve_batched: many independent problems in one persistent launch.
#include <cuda_runtime.h>

#include "internal.cuh"

extern "C" size_t osmodi_batched_workspace_bytes(int count, const osmodi_plan* plans) {
    (void)count;
    (void)plans;
    return 0;
}

extern "C" osmodi_status osmodi_solve_batched(int count, const osmodi_plan* plans, const void* const* grads, int grad_dtype,
                                              void* const* ps, int p_dtype, double tol, int max_iter, void* workspace,
                                              void* stream, osmodi_result* results) {
    (void)count; (void)plans; (void)grads; (void)grad_dtype; (void)ps; (void)p_dtype; (void)tol; (void)max_iter;
    (void)workspace; (void)stream; (void)results;
    return OSMODI_E_UNSUPPORTED;
}
