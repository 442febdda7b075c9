// batch.h -- host interface of the batched persistent launch (batch.cu), used
// by the C ABI and by the request-serving runtime (serve.cpp).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "../../include/tlgb.h"

namespace tl {

struct Batch;
int batch_create(const tl_op* ops, size_t count, int32_t flags, void* stream, Batch** out);
int batch_run(Batch* b, void* stream);
int batch_destroy(Batch* b);
size_t batch_bytes(const Batch* b);
int batch_describe(const Batch* b, char* buf, size_t len);
int batch_set_variant(Batch* b, int32_t kind, int32_t variant, int64_t unit, void* stream);

// A slot owns a device descriptor table, its pinned host staging copy and a
// unit counter, so one batch can be launched without any allocation or
// synchronisation.  A slot must not be relaunched before its previous launch
// has completed.
struct Slot;
Slot* slot_create(size_t capacity);
void slot_destroy(Slot* s);
// Plans ops[0..n) and enqueues them on st: operations the persistent kernel
// takes go into one launch, the rest run through their own kernels.
int slot_launch(Slot* s, const tl_op* const* ops, size_t n, cudaStream_t st);

// Algorithmic bytes (operands + output) of one validated operation, or a
// negative TL_E* code.
long long op_bytes(const tl_op& o);

}  // namespace tl
