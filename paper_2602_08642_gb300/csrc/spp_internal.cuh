// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "spp.h"

namespace spp {

// Host-side count of kernel launches made by this library.
extern std::atomic<uint64_t> g_launches;

inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Whether launch_dependent asks for programmatic serialisation (process-wide,
// spp_set_dependent_launch).
extern std::atomic<int> g_dependent_launch;

// Test of the reconstruction's bounded waits: the tile whose copies the next
// pipelined reconstruction launch skips (-1: none; spp_test_stall_reconstruction).
extern std::atomic<int> g_recon_stall_tile;

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Streaming multiprocessor count of the current device (cached per device).
int sm_count();

// Maps the last CUDA error of a launch sequence to an SPP code.
inline int launch_status() { return cudaGetLastError() == cudaSuccess ? SPP_OK : SPP_ERR_CUDA; }

// Programmatic dependent launch (sm_90 and later).  A kernel launched by
// launch_dependent may be scheduled while the kernel before it in the stream
// is still running; pdl_wait() returns once that kernel has completed and its
// memory operations are visible, so every such kernel calls it before its
// first global load or store.  pdl_trigger() allows the next kernel's blocks
// to be scheduled; called after pdl_wait(), at most two kernels of a stream
// are resident at a time.  Both are no-ops in a kernel launched normally.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches kernel<<<grid, block, smem, stream>>>(args...) with programmatic
// stream serialisation, so that its launch and prologue overlap the end of
// the previous kernel in the stream; falls back to a plain launch if the
// attribute is refused.
template <typename... KArgs, typename... Args>
inline void launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t stream, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    if (g_dependent_launch.load(std::memory_order_relaxed)) {
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...) == cudaSuccess) return;
        (void)cudaGetLastError();
        cfg.numAttrs = 0;
    }
    (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Records a device-side error: the first one wins.
__device__ __forceinline__ void set_status(int32_t *status, int code) {
    if (status) atomicCAS(reinterpret_cast<int *>(status), 0, code);
}

// SplitMix64 (Steele, Lea & Flood 2014): golden gamma and output mix.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Stream key of (seed, frame); element i of the stream is mix(key + (i+1) gamma).
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint32_t frame) {
    return mix64(seed + (static_cast<uint64_t>(frame) + 1ull) * kGamma);
}

__host__ __device__ __forceinline__ uint64_t stream_bits(uint64_t key, uint64_t i) {
    return mix64(key + (i + 1ull) * kGamma);
}

}  // namespace spp
