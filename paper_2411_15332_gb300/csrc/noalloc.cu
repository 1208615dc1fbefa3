// Readouts for callers that must not allocate device memory.
//
// mera_observables() keeps its per-block partial sums in a small scratch
// buffer that the state allocates with cudaMalloc.  Some callers cannot let
// a library call cudaMalloc: a framework whose caching allocator owns all
// device memory, or a latency-critical loop that cannot afford the implicit
// device synchronisation cudaMalloc / cudaFree may cause.  This file gives
// them the same reduction with the scratch in a fixed device array.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "reduce.cuh"

namespace mera {

// Partial sums of the fixed reduction partition: at most 1024 blocks, three
// sums each, plus the three results.  Every GPU that loads the library keeps
// this array (24.6 KB) until the process exits.
static constexpr int NOALLOC_MAX_BLOCKS = 1024;
static __device__ __align__(256) double g_noalloc_scratch[3 * NOALLOC_MAX_BLOCKS + 8];

// Device address of the array, looked up once per device with that device
// current (in host code the symbol's name is only a stand-in).
static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[128];

static int noalloc_scratch(double** out) {
    int dev = 0;
    MERA_CHECK_CUDA(cudaGetDevice(&dev));
    MERA_RETURN_IF(dev < 0 || dev >= 128, MERA_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error("cudaGetSymbolAddress(scratch) on device %d: %s", dev, cudaGetErrorString(e));
            return MERA_ECUDA;
        }
        g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[dev];
    return MERA_OK;
}

}  // namespace mera

using namespace mera;

extern "C" int mera_observables_noalloc(const void* dev_psi, int n, int dtype, int q, void* stream, double out[3]) {
    try {
        MERA_RETURN_IF(dev_psi == nullptr || out == nullptr, MERA_EINVAL, "NULL argument");
        MERA_RETURN_IF(n < 1 || n > MERA_MAX_QUBITS, MERA_EINVAL,
                       "n=%d outside [1, %d], the sizes the fixed scratch array serves", n, MERA_MAX_QUBITS);
        MERA_RETURN_IF(dtype != MERA_C64 && dtype != MERA_C128, MERA_EUNSUPPORTED, "unknown dtype %d", dtype);
        MERA_RETURN_IF(q < 0 || q >= n, MERA_EINVAL, "qubit %d out of range", q);
        MERA_RETURN_IF(((uintptr_t)dev_psi & 15) != 0, MERA_EINVAL, "dev_psi must be 16-byte aligned");
        const int nb = reduce_blocks(1ull << n);
        MERA_RETURN_IF(nb > NOALLOC_MAX_BLOCKS, MERA_EINVAL, "reduction needs %d partial sums, the array holds %d", nb,
                       NOALLOC_MAX_BLOCKS);
        double* scratch = nullptr;
        MERA_TRY(noalloc_scratch(&scratch));
        // a view of the caller's amplitudes; nothing is allocated
        mera_state view;
        view.data = const_cast<void*>(dev_psi);
        view.n = n;
        view.dtype = dtype;
        view.stream = (cudaStream_t)stream;
        // every block overwrites the partials that the final step reads, so
        // nothing has to be cleared between calls
        MERA_TRY(observables_device(&view, q, scratch, scratch + 3 * NOALLOC_MAX_BLOCKS));
        MERA_CHECK_CUDA(cudaMemcpyAsync(out, scratch + 3 * NOALLOC_MAX_BLOCKS, 3 * sizeof(double),
                                        cudaMemcpyDeviceToHost, view.stream));
        MERA_CHECK_CUDA(cudaStreamSynchronize(view.stream));
        return MERA_OK;
    } catch (...) {
        set_error("unexpected C++ exception");
        return MERA_EINVAL;
    }
}
