// hs_device.cuh -- device-side helpers shared by the libhs kernels:
// candidate records, warp-aggregated append, mbarrier/TMA wrappers with
// bounded waits, and compile-time loops.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <utility>

#include "../../include/hs.h"

namespace hs {

// ---- compile-time loop ------------------------------------------------------

template <int B, typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, B + I>{}), ...);
}

// Calls f(std::integral_constant<int, i>) for i = B .. E-1, fully unrolled.
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (E > B)
        static_for_impl<B>(static_cast<F &&>(f), std::make_integer_sequence<int, E - B>{});
}

// ---- element conversion --------------------------------------------------------

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

// ---- candidate records ---------------------------------------------------------

// One 16-byte record {bin, z | k<<16 | flags<<24, power, 0}, the hs_cand layout.
__device__ __forceinline__ void put_record(hs_cand *rec, uint32_t idx, uint32_t cap,
                                           uint32_t bin, int z, int k, uint32_t flags,
                                           float power)
{
    if (idx >= cap)
        return;
    uint4 v;
    v.x = bin;
    v.y = (uint32_t)(uint16_t)(int16_t)z | ((uint32_t)k << 16) | (flags << 24);
    v.z = __float_as_uint(power);
    v.w = 0u;
    reinterpret_cast<uint4 *>(rec)[idx] = v;
}

// Warp-aggregated reservation of n_lane record slots per lane: a ballot per
// bit of n_lane gives each lane the exclusive prefix of the counts below it,
// and one lane does a single atomicAdd for the warp's total.  Every lane of
// the warp must call it (n_lane may be 0).  Returns the lane's first slot.
__device__ __forceinline__ uint32_t warp_reserve(uint32_t *counter, uint32_t n_lane)
{
    const unsigned full = 0xffffffffu;
    const unsigned any = __ballot_sync(full, n_lane != 0u);
    if (any == 0u)
        return 0u;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    uint32_t prefix = 0u, total = 0u;
#pragma unroll
    for (int b = 0; b < 7; ++b) { // n_lane <= 64
        const unsigned bal = __ballot_sync(full, (n_lane >> b) & 1u);
        prefix += (uint32_t)__popc(bal & below) << b;
        total += (uint32_t)__popc(bal) << b;
    }
    const int leader = __ffs(any) - 1;
    uint32_t base = 0u;
    if ((int)lane == leader)
        base = atomicAdd(counter, total);
    base = __shfl_sync(full, base, leader);
    return base + prefix;
}

__device__ __forceinline__ void set_status(uint32_t *counters, uint32_t s)
{
    atomicCAS(counters + 1, 0u, s);
}

// ---- timing, mbarrier and TMA (inline PTX, sm_90+ forms valid on sm_103a) -------

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return done != 0u;
}

// Plain arrival (no transaction bytes) on a barrier.
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Named barrier `id` (1..15) over `count` threads (a multiple of 32): every
// participating thread gets the OR of `v` over the group.
__device__ __forceinline__ bool group_or(int id, int count, bool v)
{
    uint32_t r;
    __syncwarp();
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id), "r"(count)
                 : "memory");
    return r != 0u;
}

__device__ __forceinline__ void group_sync(int id, int count)
{
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// One test of phase `parity` that may suspend the thread for up to hint_ns
// until the phase completes (the hardware may return earlier).
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity), "r"(hint_ns)
                 : "memory");
    return done != 0u;
}

// The retry loop of mbar_wait_bounded, out of line so the waiting thread's
// straight-line code carries no loop.
static __device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait_hint(bar, parity, 100000u)) {
        if (globaltimer_ns() - t0 > limit_ns)
            return false;
    }
    return true;
}

// Wait for phase `parity` of the barrier for at most limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns)
{
    if (mbar_try_wait_hint(bar, parity, 1000000u)) // usually completes here
        return true;
    return mbar_wait_slow(bar, parity, limit_ns);
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y,
                                            uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

// Prefetch a 2-D box into L2 (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_l2_2d(const void *tmap, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const void *tmap)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

} // namespace hs
