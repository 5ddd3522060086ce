// Split-precision tensor-core path: not built yet; every shape reports
// "unsupported" so the caller uses the FP64 kernel.
#include "common.cuh"

int launch_zgemm_split(const GemmArgs&, cudaStream_t, void*, size_t) { return -1; }
size_t split_workspace_bytes(const GemmArgs&) { return 0; }
