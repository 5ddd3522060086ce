// Allocation-free complex contraction for callers that cannot allocate
// device memory: code that runs while another component owns every
// allocation (a host application with its own memory pool or a fixed memory
// budget), or that must not call cudaMalloc/cudaFree at that point because
// those calls synchronise the device.  The caller passes device pointers for
// the inputs and the output; the packed split-precision operands live in one
// file-scope device array of fixed size, which every GPU that loads this
// library holds until the process exits.
#include "common.cuh"
#include "../../include/ttn.h"

#include <cstring>
#include <mutex>

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;   // 8 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached.
void* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

ttn_status scratch_for_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return TTN_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return TTN_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TTN_OK;
}

}  // namespace

extern "C" ttn_status ttn_contract_split_noalloc(const double* A, const double* B, double* C, int M, int N, int K,
                                                 void* stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1) return TTN_ERR_ARG;
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = M; g.N = N; g.Ki = K; g.Ko = 1; g.Bi = 1; g.Bo = 1;
    g.A = reinterpret_cast<const cplx*>(A); g.a_m = 1; g.a_ki = M;
    g.B = reinterpret_cast<const cplx*>(B); g.b_ki = 1; g.b_n = K;
    g.C = reinterpret_cast<cplx*>(C); g.c_m = 1; g.c_n = M;
    g.alpha = make_double2(1.0, 0.0);
    g.beta = make_double2(0.0, 0.0);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t need = split_workspace_bytes(g, 1);   // no split-K: the scratch size rule stays as documented
    if (need > NOALLOC_SCRATCH_BYTES) return TTN_ERR_ARG;   // beyond the fixed scratch
    void* scratch = nullptr;
    int packed = -1;
    if (need > 0) {
        ttn_status st = scratch_for_current_device(&scratch);
        if (st != TTN_OK) return st;
        // the error flag at the start of the scratch must start at zero
        if (cudaMemsetAsync(scratch, 0, sizeof(int), s) != cudaSuccess) return TTN_ERR_CUDA;
        packed = launch_split_pack(g, s, scratch, NOALLOC_SCRATCH_BYTES, 1);
        if (packed == -2) return TTN_ERR_ARG;
    }
    if (packed < 0) {
        // too small for the tensor-core tiles, or no tensor-map encoder in
        // this driver: the FP64 kernel needs no scratch
        launch_zgemm_f64(g, s);
        if (cudaGetLastError() != cudaSuccess) return TTN_ERR_CUDA;
        return cudaStreamSynchronize(s) == cudaSuccess ? TTN_OK : TTN_ERR_CUDA;
    }
    if (launch_split_mma(g, s, scratch, NOALLOC_SCRATCH_BYTES, 1) < 0) return TTN_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return TTN_ERR_CUDA;
    // a pipeline wait that gave up sets the first word of the scratch: read
    // it once the contraction is done, and clear it for the next call
    int flag = 0;
    if (cudaMemcpyAsync(&flag, scratch, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TTN_ERR_CUDA;
    if (flag) {
        if (cudaMemsetAsync(scratch, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return TTN_ERR_CUDA;
        return TTN_ERR_TIMEOUT;
    }
    return TTN_OK;
}
