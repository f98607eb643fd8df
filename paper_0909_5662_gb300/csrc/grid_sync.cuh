// grid_sync.cuh -- grid-wide barrier for cooperative launches, with a bounded wait.
#pragma once
#include <cstdint>

#include "ptx.cuh"

namespace dmrg {

// Zeroed before the launch that uses it.
struct GridBarrier {
    unsigned count, gen;
    int abort, pad;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every block of a cooperative launch (all resident by construction) calls it with its
// own generation counter, starting at 0.  The wait is bounded: on expiry it records the
// timeout in *status and raises the abort flag, and every block returns false (blocks
// still on their way see the flag at the barrier and return too), so the caller returns.
__device__ inline bool grid_barrier(GridBarrier* b, unsigned& gen_seen, uint64_t timeout_ns,
                                    unsigned* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = gen_seen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            uint32_t spins = 0;
            while (ld_acquire_gpu(&b->gen) == g) {
                if ((++spins & 31u) == 0) {
                    if (*reinterpret_cast<volatile int*>(&b->abort)) {
                        ok = 0;
                        break;
                    }
                    if (globaltimer_ns() - t0 > timeout_ns) {
                        atomicOr(status, DMRG_DEV_ERR_TIMEOUT);
                        atomicExch(&b->abort, 1);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        gen_seen = g + 1;
    }
    __syncthreads();
    return ok != 0;
}

// Sum over the block of one value per thread (result valid in every thread).
__device__ inline double block_sum_all(double v) {
    __shared__ double part[32];
    __shared__ double total;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) total = s;
    }
    __syncthreads();
    return total;
}

}  // namespace dmrg
