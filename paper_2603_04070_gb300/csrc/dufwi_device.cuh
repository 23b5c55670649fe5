// dufwi_device.cuh -- device primitives shared by the step kernels: shared-memory addresses,
// mbarriers, TMA tile loads (cp.async.bulk.tensor), L2 cache hints, programmatic dependent launch,
// bounded waits, the device status word, and the geometry of the padded grid of one map.
#pragma once

#include "dufwi_internal.h"

#include "../../include/dufwi.h"

namespace dufwi {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Orders this thread's earlier accesses (generic proxy) before later TMA (async proxy) accesses.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void raise_status(int *status, int code)
{
    if (status) atomicMax(status, code);
}

__device__ __forceinline__ float4 ld4s(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void st4s(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// Depth (in cells, 0..P) into the absorbing layer of padded index i along an axis of N cells.
__device__ __forceinline__ int layer_depth(int i, int P, int N)
{
    const int d = i < P ? P - i : (i > P + N - 1 ? i - (P + N - 1) : 0);
    return d < P ? d : P;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y, int z,
                                            int w)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// L2 eviction hints for the history stream (written once by the forward or recompute sweep, read
// once by the adjoint): evict-first, so that it does not push out of L2 the fields, kappa' and
// the imaging sums that every step re-reads. Build-time knob DUFWI_L2_HINTS (1 default, 0 off);
// the hints change timing only.
#ifndef DUFWI_L2_HINTS
#define DUFWI_L2_HINTS 1
#endif

__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tma_load_4d_stream(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y,
                                                   int z, int w)
{
#if DUFWI_L2_HINTS
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar)),
        "l"(l2_evict_first_policy())
        : "memory");
#else
    tma_load_4d(dst, tm, bar, x, y, z, w);
#endif
}

__device__ __forceinline__ void st4_stream(float *p, float4 v)
{
#if DUFWI_L2_HINTS
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(l2_evict_first_policy())
                 : "memory");
#else
    st4(p, v);
#endif
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *tm)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// Programmatic dependent launch: wait for the previous kernel in the stream (and its memory),
// and allow the next one to be scheduled while this one drains.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Bounded wait on an mbarrier phase: try_wait with a suspend-time hint (the thread sleeps until
// the phase completes or the hint elapses), abandoned after kWaitLimitNs of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait_sleep(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait_sleep(bar, parity)) {
        if (global_ns() - t0 > kWaitLimitNs) return false;
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ float4 fma4(float4 a, float4 b, float4 c)
{
    const float2 lo = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y));
    const float2 hi = __ffma2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w), make_float2(c.z, c.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Physical and padded size of the grid of one map (uniform calls: the problem's grid; sized
// calls: the map's own grid, inside the envelope buffers).
struct MapGrid {
    int Nx, Nz, nxp, nzp;
};

__device__ __forceinline__ MapGrid map_grid(const StepParams &p, int map)
{
    MapGrid g;
    if (p.map_dims) {
        const int2 d = __ldg(p.map_dims + map);
        g.Nx = d.x;
        g.Nz = d.y;
        g.nxp = d.x + 2 * p.P;
        g.nzp = d.y + 2 * p.P;
    } else {
        g.Nx = p.Nx;
        g.Nz = p.Nz;
        g.nxp = p.nxp;
        g.nzp = p.nzp;
    }
    return g;
}

// Is the region [x0, x0 + w) x [z0, z0 + h) (clipped to the padded grid) free of damping?
__device__ __forceinline__ bool region_interior(const StepParams &p, const MapGrid &g, int x0, int z0, int w, int h)
{
    return x0 >= p.P && min(x0 + w, g.nxp) <= p.P + g.Nx && z0 >= p.P && min(z0 + h, g.nzp) <= p.P + g.Nz;
}

}  // namespace
}  // namespace dufwi
