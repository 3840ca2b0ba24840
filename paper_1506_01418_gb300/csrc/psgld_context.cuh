// psgld_context.cuh -- context creation with a given allocator, shared by
// the C API (psgld_create) and the serving loop (psgld_server.cu).
#pragma once

#include "psgld_internal.cuh"

namespace psgld {

// psgld_create with the context's allocator given (nullptr: the one set by
// psgld_set_allocator, else cudaMalloc / cudaFree).
psgld_status create_context(int64_t I, int64_t J, int32_t K, int32_t B, double tweedie_p, double phi,
                            const psgld_prior *prior, const psgld_allocator *allocator, psgld_ctx **out);

}  // namespace psgld
