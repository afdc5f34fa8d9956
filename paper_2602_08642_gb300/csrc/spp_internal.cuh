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

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Streaming multiprocessor count of the current device (cached per device).
int sm_count();

// Maps the last CUDA error of a launch sequence to an SPP code.
inline int launch_status() { return cudaGetLastError() == cudaSuccess ? SPP_OK : SPP_ERR_CUDA; }

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
