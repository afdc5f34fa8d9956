// Status codes, launch counter and small utilities of the C ABI.
#include <mutex>

#include "spp_internal.cuh"
#include "tma_host.cuh"

namespace spp {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_dependent_launch{1};
std::atomic<int> g_recon_stall_tile{-1};

int sm_count() {
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 152;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 152;
    if (dev < 64) cache[dev] = n;
    return n;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace spp

extern "C" {

const char *spp_strerror(int code) {
    switch (code) {
        case SPP_OK: return "ok";
        case SPP_ERR_ARG: return "bad argument (null pointer or size out of range)";
        case SPP_ERR_ALIGN: return "pointer not 16-byte aligned";
        case SPP_ERR_SHAPE: return "W or H not divisible by 2^(L-1), or L outside [2, 5]";
        case SPP_ERR_WORKSPACE: return "workspace too small";
        case SPP_ERR_CAPACITY: return "more samples than the sample buffers hold";
        case SPP_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        case SPP_ERR_INPUT: return "density has NaN, inf or negative values, or sums to zero";
        case SPP_ERR_CUDA: return "CUDA runtime error";
        default: return "unknown status code";
    }
}

int spp_abi_version(void) { return 7; }

uint64_t spp_launch_count(void) { return spp::g_launches.load(std::memory_order_relaxed); }

int spp_set_dependent_launch(int on) { return spp::g_dependent_launch.exchange(on ? 1 : 0); }

int spp_get_dependent_launch(void) { return spp::g_dependent_launch.load(); }

int spp_test_stall_reconstruction(int tile) {
    if (tile < -1) return SPP_ERR_ARG;
    spp::g_recon_stall_tile.store(tile);
    return SPP_OK;
}

int spp_get_status(const int32_t *status, cudaStream_t stream) {
    if (!status) return SPP_ERR_ARG;
    int32_t host = 0;
    if (cudaMemcpyAsync(&host, status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) !=
        cudaSuccess)
        return SPP_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return SPP_ERR_CUDA;
    return host;
}

int spp_clear_status(int32_t *status, cudaStream_t stream) {
    if (!status) return SPP_ERR_ARG;
    return cudaMemsetAsync(status, 0, sizeof(int32_t), stream) == cudaSuccess ? SPP_OK
                                                                              : SPP_ERR_CUDA;
}

}  // extern "C"
