// Host-callable launchers of the library's kernels (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "eg_internal.cuh"

namespace eg {

// Steps (a)+(c): gradient pointers into lab, critical-vertex records, counts.
cudaError_t launch_classify_d(int d, const FieldDev *fields, int nf, uint64_t total_bricks,
                              cudaStream_t st);

// Step (b): labels = fixed points of the gradient pointers.
cudaError_t launch_resolve(const FieldDev *fields, int nf, uint64_t total_bricks, cudaStream_t st);

// Steps (d)+(e): arcs and the sorted CSR graph.  ws: zeroed workspace of
// emit_workspace_bytes(total_bricks) bytes.
size_t emit_workspace_bytes(uint64_t total_bricks);
cudaError_t launch_emit_d(int d, const FieldDev *fields, int nf, uint64_t total_bricks, void *ws,
                          int sm_count, cudaStream_t st);

}  // namespace eg
