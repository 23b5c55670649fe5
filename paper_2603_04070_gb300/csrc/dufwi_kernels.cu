// dufwi_kernels.cu -- sm_103a kernels of the damped acoustic simulator (Eq. 2) and of its
// discrete adjoint with the zero-lag imaging condition (Eq. 6).
//
// The step kernel serves both directions. For the stepper of Eq. 2,
//   U^{n+1} = a U^n + b U^{n-1} + kappa' L U^n + s^n,   L = unscaled central stencil,
// the exact adjoint of the recursion, written for mu = kappa' * lambda, is
//   mu^m = a mu^{m+1} + b mu^{m+2} + kappa' L mu^{m+1} + kappa'_r q^m_r,
// which is the same update (L is symmetric with a zero exterior). The gradient is then
//   dJ/dC = (2/C) sum_m mu^m * L U^{m-1},
// since dkappa'/dC = 2 kappa'/C. One kernel body therefore handles the forward sweep, the
// recompute sweep and the adjoint sweep; the variants differ only in their fused epilogue
// (receiver sampling, history write, imaging accumulation).
//
// Tile scheme: each CTA owns a 64 x 64 output tile of one shot. One TMA load brings the 72 x 72
// box of U^n (halo 4) into shared memory; out-of-range box elements read as zero, which is the
// zero exterior of the stencil. The load completes on an mbarrier. Each thread computes a
// 4 (x) x 4 (z) block from 128-bit shared-memory reads: z-neighbours come from a register
// column and x-neighbours from the adjacent float4s of the same row. Then it streams U^{n-1},
// kappa' and, in the adjoint, the history and the gradient with coalesced 128-bit global
// accesses.
#include "dufwi_internal.h"

#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

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

__device__ __forceinline__ void raise_status(int *status, int code)
{
    if (status) atomicMax(status, code);
}

__device__ __forceinline__ float4 ld4s(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void set_comp(float4 &v, int i, float s)
{
    if (i == 0) v.x = s; else if (i == 1) v.y = s; else if (i == 2) v.z = s; else v.w = s;
}

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

template <int MODE, int TZ>
struct TileLayout {
    static constexpr int kBoxRows = TZ + 2 * kHalo;
    static constexpr int kBox = kBoxX * kBoxRows;                      // U^n (or mu^{m+1}) with halo
    static constexpr int kTile = kTileX * TZ;
    static constexpr int kTiles = MODE == kAdjoint ? 4 : 2;            // prev, kappa (+ history, sums)
    static constexpr int kFloats = kBox + kTiles * kTile;
    static constexpr uint32_t kBytes = kFloats * sizeof(float);
    static constexpr int kThreadsPerCta = (kTileX / 4) * (TZ / 4);      // 4 (x) x 4 (z) outputs each
};

// One 64 x TZ output tile of one shot per CTA. A single mbarrier collects the TMA loads of the
// (64 + 8) x (TZ + 8) box of U^n and of the 64 x TZ tiles of U^{n-1} and kappa' (and, in the
// adjoint, of Lap(U^{m-1}) and of the running imaging sum). Many small CTAs stay resident per SM,
// so the loads of some overlap the arithmetic of others.
// Minimum resident CTAs of 128 threads per SM requested from the register allocator (the 64-row
// tile variant asks for half as many CTAs of 256 threads). Build-time knob.
#ifndef DUFWI_STEP_MIN_CTAS_128
#define DUFWI_STEP_MIN_CTAS_128 5
#endif

template <int R, int MODE, int TZ>
__global__ void __launch_bounds__(TileLayout<MODE, TZ>::kThreadsPerCta,
                                  (DUFWI_STEP_MIN_CTAS_128 * 128 + TileLayout<MODE, TZ>::kThreadsPerCta - 1) /
                                      TileLayout<MODE, TZ>::kThreadsPerCta)
step_kernel(const __grid_constant__ StepMaps tm, const StepParams p)
{
    using TL = TileLayout<MODE, TZ>;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;

    const int tid = threadIdx.x;
    const int s = blockIdx.z;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * TZ;
    const int tx_idx = s % p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *box = smem;
    float *pv = box + TL::kBox;
    float *kp = pv + TL::kTile;
    float *hs = kp + TL::kTile;
    float *gg = hs + TL::kTile;

    if (tid == 0) {
        prefetch_tensormap(&tm.cur_box);
        prefetch_tensormap(&tm.out_tile);
        mbar_init(&bar, 1);
    }
    __syncthreads();

    grid_dependency_wait();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, TL::kBytes);
        tma_load_3d(box, &tm.cur_box, &bar, x0 - kHalo, z0 - kHalo, s);
        tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
        tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, s / p.n_tx);
        if (MODE == kAdjoint) {
            tma_load_4d(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
            tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, s);
        }
    }
    grid_dependents_launch();

    // Receivers of this transmit inside this tile: a host-built table gives the range of them
    // (indices into rx_sorted), so no CTA scans the whole receiver list.
    int2 rx_range = make_int2(0, 0);
    if (MODE != kFwdHist) rx_range = __ldg(p.rx_tab + tx_idx * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x);
    int src_node = -1;
    if (MODE != kAdjoint) src_node = __ldg(p.inj_node + tx_idx);

    const int lx = (tid & 15) * 4;
    const int lz = (tid >> 4) * 4;
    const int gx = x0 + lx;
    const bool col_ok = gx < p.nxp;
    const bool interior = (x0 >= p.P) && (min(x0 + kTileX, p.nxp) <= p.P + p.Nx) && (z0 >= p.P) &&
                          (min(z0 + TZ, p.nzp) <= p.P + p.Nz);
    int xd[4];
    if (!interior) {
#pragma unroll
        for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, p.Nx);
    }

    // One thread polls the mbarrier; the others park on the CTA barrier and then take their own
    // (immediately successful) acquire of the completed phase.
    int fail = 0;
    if (tid == 0) fail = !mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(fail)) {
        if (tid == 0) raise_status(p.status, DUFWI_ERR_TIMEOUT);
        mbar_wait_bounded(&bar, 0);
        return;
    }
    if (!mbar_try_wait_sleep(&bar, 0) && !mbar_wait_bounded(&bar, 0)) {
        raise_status(p.status, DUFWI_ERR_TIMEOUT);
        return;
    }

    // Column window: rows lz + kHalo - R .. lz + kHalo + 3 + R of the float4 at x = lx.
    float4 col[4 + 2 * R];
#pragma unroll
    for (int i = 0; i < 4 + 2 * R; ++i) col[i] = ld4s(box + (lz + kHalo - R + i) * kBoxX + kHalo + lx);

    // The four x-lanes of a thread are processed as two packed FP32 pairs (lanes 0-1 and 2-3)
    // with the sm_100-family f32x2 instructions; every operation keeps the IEEE rounding and
    // order of the scalar formulation.
    const float2 two2 = make_float2(2.0f, 2.0f), m4 = make_float2(-4.0f, -4.0f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float *row = box + (lz + kHalo + j) * kBoxX + lx;
        const float4 lft = ld4s(row);
        const float4 rgt = ld4s(row + 8);
        const float4 ctr = col[R + j];
        const float w[12] = {lft.x, lft.y, lft.z, lft.w, ctr.x, ctr.y, ctr.z, ctr.w, rgt.x, rgt.y, rgt.z, rgt.w};
        // Laplacian in difference form, sum_k c_k ((x_{+k} + x_{-k}) + (z_{+k} + z_{-k}) - 4u):
        // exactly zero on a constant field whatever the rounding of the weights.
        float2 lap[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 u = make_float2(w[4 + 2 * h], w[5 + 2 * h]);
            const float2 nu4 = __fmul2_rn(m4, u);
            float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int kk = 1; kk <= R; ++kk) {
                const float2 xs = (kk & 1)
                    ? make_float2(w[4 + 2 * h - kk] + w[4 + 2 * h + kk], w[5 + 2 * h - kk] + w[5 + 2 * h + kk])
                    : __fadd2_rn(make_float2(w[4 + 2 * h - kk], w[5 + 2 * h - kk]),
                                 make_float2(w[4 + 2 * h + kk], w[5 + 2 * h + kk]));
                const float4 &cm = col[R + j - kk], &cp = col[R + j + kk];
                const float2 zs = h == 0 ? __fadd2_rn(make_float2(cm.x, cm.y), make_float2(cp.x, cp.y))
                                         : __fadd2_rn(make_float2(cm.z, cm.w), make_float2(cp.z, cp.w));
                const float2 t = __fadd2_rn(__fadd2_rn(xs, zs), nu4);
                acc = __ffma2_rn(make_float2(p.c[kk], p.c[kk]), t, acc);
            }
            lap[h] = acc;
        }

        const int gz = z0 + lz + j;
        if (!col_ok || gz >= p.nzp) continue;
        const int lo = (lz + j) * kTileX + lx;
        const float4 prev = ld4s(pv + lo);
        const float4 kap = ld4s(kp + lo);
        const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;

        // U^{n+1} = 2u - p + (a - 2) u + (b + 1) p + kappa' L, with the small damping terms
        // a - 2 = -q (2 + q)/(1 + q) and b + 1 = 2q/(1 + q), q = D dt, read from a table over
        // the layer depths (computed in FP64 on the host, rounded once).
        float2 base[2];
        base[0] = __ffma2_rn(two2, make_float2(ctr.x, ctr.y), make_float2(-prev.x, -prev.y));
        base[1] = __ffma2_rn(two2, make_float2(ctr.z, ctr.w), make_float2(-prev.z, -prev.w));
        if (!interior) {
            const float2 *trow = p.damp_tab + layer_depth(gz, p.P, p.Nz) * (p.P + 1);
            const float2 t0 = __ldg(trow + xd[0]), t1 = __ldg(trow + xd[1]);
            const float2 t2 = __ldg(trow + xd[2]), t3 = __ldg(trow + xd[3]);
            base[0] = __ffma2_rn(make_float2(t0.x, t1.x), make_float2(ctr.x, ctr.y),
                                 __ffma2_rn(make_float2(t0.y, t1.y), make_float2(prev.x, prev.y), base[0]));
            base[1] = __ffma2_rn(make_float2(t2.x, t3.x), make_float2(ctr.z, ctr.w),
                                 __ffma2_rn(make_float2(t2.y, t3.y), make_float2(prev.z, prev.w), base[1]));
        }
        const float2 n01 = __ffma2_rn(make_float2(kap.x, kap.y), lap[0], base[0]);
        const float2 n23 = __ffma2_rn(make_float2(kap.z, kap.w), lap[1], base[1]);
        float4 nxt = make_float4(n01.x, n01.y, n23.x, n23.y);
        float4 lp = make_float4(lap[0].x, lap[0].y, lap[1].x, lap[1].y);
        // Lanes past the last column stay zero (they are padding of the row pitch).
        if (gx + 4 > p.nxp) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (gx + i >= p.nxp) { set_comp(nxt, i, 0.f); set_comp(lp, i, 0.f); }
        }
        st4(p.out + o, nxt);
        if (MODE == kFwdSampleHist || MODE == kFwdHist) st4(p.hist + o, lp);
        if (MODE == kAdjoint) {
            const float4 hv = ld4s(hs + lo);
            const float4 gv = ld4s(gg + lo);
            const float2 g01 = __ffma2_rn(make_float2(nxt.x, nxt.y), make_float2(hv.x, hv.y), make_float2(gv.x, gv.y));
            const float2 g23 = __ffma2_rn(make_float2(nxt.z, nxt.w), make_float2(hv.z, hv.w), make_float2(gv.z, gv.w));
            st4(p.grad + o, make_float4(g01.x, g01.y, g23.x, g23.y));
        }
    }

    // Receiver sampling of U^n from the box (each receiver lies in exactly one tile); placed
    // after the arithmetic so the table load is long complete.
    if (MODE == kFwdSample || MODE == kFwdSampleHist) {
        for (int e = tid; e < rx_range.y; e += TL::kThreadsPerCta) {
            const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
            const int node = __ldg(p.smp_node + tx_idx * p.n_rx + r);
            const int zn = node >> 16, xn = node & 0xffff;
            p.cd[(static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r] =
                box[(zn - z0 + kHalo) * kBoxX + (xn - x0 + kHalo)];
        }
    }

    // Point injections into the just-written cells of this tile (the CTA is their only writer,
    // so after the barrier an atomic add is race-free and sees the stored value).
    if (MODE == kAdjoint) {
        if (rx_range.y == 0) return;
        __syncthreads();
        for (int e = tid; e < rx_range.y; e += TL::kThreadsPerCta) {
            const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
            const int node = __ldg(p.inj_node + tx_idx * p.n_rx + r);
            const int zn = node >> 16, xn = node & 0xffff;
            const long long o = shot_off + static_cast<long long>(zn) * p.pitch + xn;
            const float v = __ldg(p.inj_val + (static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r);
            atomicAdd(p.out + o, v);
            atomicAdd(p.grad + o, v * hs[(zn - z0) * kTileX + (xn - x0)]);
        }
    } else {
        const bool has_src = (src_node >> 16) >= z0 && (src_node >> 16) < z0 + TZ && (src_node & 0xffff) >= x0 &&
                             (src_node & 0xffff) < x0 + kTileX;
        if (!has_src) return;
        __syncthreads();
        if (tid == 0) {
            const long long o = shot_off + static_cast<long long>(src_node >> 16) * p.pitch + (src_node & 0xffff);
            const float wv = __ldg(p.inj_val + static_cast<long long>(p.wav_per_tx ? tx_idx : 0) * p.nt + p.step);
            atomicAdd(p.out + o, p.inj_scale * wv);
        }
    }
}

// kappa' = C^2 (dt/dx)^2 / (1 + D dt) on the padded grid; C extended by edge replication.
__global__ void setup_kappa_kernel(const float *sos, const float *density, float *kap, int *status, int Nx,
                                   int Nz, int P, int nxp, int nzp, int pitch, double r2, double d0, double dt,
                                   double c_max)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int b = blockIdx.z;
    if (x >= pitch) return;
    float *dst = kap + (static_cast<long long>(b) * nzp + z) * pitch + x;
    if (x >= nxp) { *dst = 0.f; return; }
    const int xs = min(max(x - P, 0), Nx - 1), zs = min(max(z - P, 0), Nz - 1);
    const long long src = (static_cast<long long>(b) * Nz + zs) * Nx + xs;
    const double C = sos[src];
    if (!isfinite(C)) raise_status(status, DUFWI_ERR_NONFINITE);
    else if (!(C > 0.0) || C > c_max) raise_status(status, DUFWI_ERR_CFL);
    if (density && x >= P && x < P + Nx && z >= P && z < P + Nz) {
        if (density[src] != density[static_cast<long long>(b) * Nz * Nx]) raise_status(status, DUFWI_ERR_UNSUPPORTED);
    }
    const int dxl = x < P ? P - x : (x > P + Nx - 1 ? x - (P + Nx - 1) : 0);
    const int dzl = z < P ? P - z : (z > P + Nz - 1 ? z - (P + Nz - 1) : 0);
    const double xx = static_cast<double>(dxl) / P, zz = static_cast<double>(dzl) / P;
    const double D = d0 * xx * xx + d0 * zz * zz;
    *dst = static_cast<float>(C * C * r2 / (1.0 + D * dt));
}

__global__ void sample_kernel(const float *field, const int *rx_node, float *cd, long long slice, int pitch,
                              int n_tx, int n_rx, int nt, int step)
{
    const int s = blockIdx.x;
    const int tx_idx = s % n_tx;
    for (int r = threadIdx.x; r < n_rx; r += blockDim.x) {
        const int node = rx_node[tx_idx * n_rx + r];
        cd[(static_cast<long long>(s) * nt + step) * n_rx + r] =
            field[s * slice + static_cast<long long>(node >> 16) * pitch + (node & 0xffff)];
    }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// Residual of one shot: J partial (FP64, fixed order) and the scaled adjoint source
// kappa'_r * 2 (M_sim - M_obs).
__global__ void residual_kernel(const float *cd_sim, const float *cd_obs, const float *kap, const int *rx_node,
                                float *asrc, double *partial, int *status, int n_tx, int n_rx, int nt,
                                long long slice, int pitch)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    const int tx_idx = s % n_tx, map = s / n_tx;
    const long long base = static_cast<long long>(s) * nt * n_rx;
    const long long n = static_cast<long long>(nt) * n_rx;
    double acc = 0.0;
    bool bad = false;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const int r = static_cast<int>(i % n_rx);
        const float obs = cd_obs[base + i];
        if (!isfinite(obs)) bad = true;
        const float d = cd_sim[base + i] - obs;
        acc += static_cast<double>(d) * static_cast<double>(d);
        const int node = rx_node[tx_idx * n_rx + r];
        const float kr = kap[map * slice + static_cast<long long>(node >> 16) * pitch + (node & 0xffff)];
        asrc[base + i] = kr * (2.0f * d);
    }
    if (bad) raise_status(status, DUFWI_ERR_NONFINITE);
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) partial[s] = t;
}

__global__ void misfit_sum_kernel(const double *partial, double *misfit, int n_maps, int n_tx)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_maps) return;
    double J = 0.0;
    for (int t = 0; t < n_tx; ++t) J += partial[b * n_tx + t];
    misfit[b] = J;
}

// Fold of the padded per-shot imaging sums onto the physical grid with the FP64 reduction over
// transmits, in two short passes (every dependent FP64 chain stays below n_tx (P + 1) terms):
//   fold_x: F[b][zp][ix] = sum_tx sum_{xp copying ix} G_s[zp][xp]
//   fold_z: g[b][iz][ix] = (2 / C) sum_{zp copying iz} F[b][zp][ix]
__global__ void fold_x_kernel(const float *g_shot, double *fx, int n_tx, int Nx, int P, int nzp, long long slice,
                              int pitch)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int zp = blockIdx.y;
    const int b = blockIdx.z;
    if (ix >= Nx) return;
    const int xlo = ix == 0 ? 0 : ix + P, xhi = ix == Nx - 1 ? Nx + 2 * P - 1 : ix + P;
    double acc = 0.0;
    for (int t = 0; t < n_tx; ++t) {
        const float *g = g_shot + static_cast<long long>(b * n_tx + t) * slice + static_cast<long long>(zp) * pitch;
        for (int x = xlo; x <= xhi; ++x) acc += g[x];
    }
    fx[(static_cast<long long>(b) * nzp + zp) * Nx + ix] = acc;
}

__global__ void fold_z_kernel(const double *fx, const float *sos, float *grad, int Nx, int Nz, int P, int nzp)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int b = blockIdx.z;
    if (ix >= Nx) return;
    const int zlo = iz == 0 ? 0 : iz + P, zhi = iz == Nz - 1 ? Nz + 2 * P - 1 : iz + P;
    double acc = 0.0;
    for (int z = zlo; z <= zhi; ++z) acc += fx[(static_cast<long long>(b) * nzp + z) * Nx + ix];
    const long long o = (static_cast<long long>(b) * Nz + iz) * Nx + ix;
    grad[o] = static_cast<float>(acc * (2.0 / static_cast<double>(sos[o])));
}

// ---- checkpoint snapshots -------------------------------------------------------------------
// Compressed snapshots store U^n and U^n - U^{n-1}, each scaled by a power of two 2^-e with
// 2^(e-1) <= max|.| < 2^e (exact in FP32), times 2^14 for FP16 so that the range sits well
// inside FP16's normal numbers.
__device__ __forceinline__ float snap_mult(unsigned bits, int dtype)
{
    const float m = __uint_as_float(bits);
    if (!(m > 0.f)) return 0.f;
    const int e = ilogbf(m) + 1;
    return ldexpf(1.0f, (dtype == DUFWI_SNAP_FP16 ? 14 : 0) - e);
}

__global__ void snap_absmax_kernel(const float *cur, const float *prev, unsigned *scale_bits, long long slice)
{
    __shared__ float red[2][32];
    const int s = blockIdx.y;
    const float4 *a = reinterpret_cast<const float4 *>(cur + s * slice);
    const float4 *b = reinterpret_cast<const float4 *>(prev + s * slice);
    float mu = 0.f, md = 0.f;
    for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < slice / 4; i += (long long)gridDim.x * blockDim.x) {
        const float4 u = a[i], v = b[i];
        mu = fmaxf(mu, fmaxf(fmaxf(fabsf(u.x), fabsf(u.y)), fmaxf(fabsf(u.z), fabsf(u.w))));
        md = fmaxf(md, fmaxf(fmaxf(fabsf(u.x - v.x), fabsf(u.y - v.y)), fmaxf(fabsf(u.z - v.z), fabsf(u.w - v.w))));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = mu; red[1][w] = md; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { mu = fmaxf(mu, red[0][i]); md = fmaxf(md, red[1][i]); }
        mu = fmaxf(mu, red[0][0]); md = fmaxf(md, red[1][0]);
        atomicMax(scale_bits + 2 * s, __float_as_uint(mu));
        atomicMax(scale_bits + 2 * s + 1, __float_as_uint(md));
    }
}

template <typename T> __device__ __forceinline__ T to_t(float v);
template <> __device__ __forceinline__ __nv_bfloat16 to_t<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half to_t<__half>(float v) { return __float2half_rn(v); }
__device__ __forceinline__ float from_t(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float from_t(__half v) { return __half2float(v); }

template <typename T>
__global__ void snap_store_kernel(const float *cur, const float *prev, T *su, T *sd, const unsigned *scale_bits,
                                  int dtype, long long slice)
{
    const int s = blockIdx.y;
    const float mu = snap_mult(scale_bits[2 * s], dtype), md = snap_mult(scale_bits[2 * s + 1], dtype);
    const long long off = s * slice;
    for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < slice; i += (long long)gridDim.x * blockDim.x) {
        const float u = cur[off + i], v = prev[off + i];
        su[off + i] = to_t<T>(u * mu);
        sd[off + i] = to_t<T>((u - v) * md);
    }
}

template <typename T>
__global__ void snap_load_kernel(float *cur, float *prev, const T *su, const T *sd, const unsigned *scale_bits,
                                 int dtype, long long slice)
{
    const int s = blockIdx.y;
    const float mu = snap_mult(scale_bits[2 * s], dtype), md = snap_mult(scale_bits[2 * s + 1], dtype);
    const float iu = mu > 0.f ? 1.0f / mu : 0.f, id = md > 0.f ? 1.0f / md : 0.f;
    const long long off = s * slice;
    for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < slice; i += (long long)gridDim.x * blockDim.x) {
        const float u = from_t(su[off + i]) * iu;
        const float d = from_t(sd[off + i]) * id;
        cur[off + i] = u;
        prev[off + i] = u - d;
    }
}

}  // namespace

// ---- launchers ------------------------------------------------------------------------------

template <int R, int MODE, int TZ>
static cudaError_t launch_step_rmt(const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    using TL = TileLayout<MODE, TZ>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<R, MODE, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TL::kBytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(step_kernel<R, MODE, TZ>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + TZ - 1) / TZ, p.n_maps * p.n_tx);
    cfg.blockDim = dim3(TL::kThreadsPerCta);
    cfg.dynamicSmemBytes = TL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step_kernel<R, MODE, TZ>, tm, p);
}

template <int R, int MODE>
static cudaError_t launch_step_rm(const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    switch (p.tile_z) {
    case 32: return launch_step_rmt<R, MODE, 32>(tm, p, st);
    case 64: return launch_step_rmt<R, MODE, 64>(tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R>
static cudaError_t launch_step_r(int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_step_rm<R, kFwdSample>(tm, p, st);
    case kFwdSampleHist: return launch_step_rm<R, kFwdSampleHist>(tm, p, st);
    case kFwdHist: return launch_step_rm<R, kFwdHist>(tm, p, st);
    case kAdjoint: return launch_step_rm<R, kAdjoint>(tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    switch (radius) {
    case 1: return launch_step_r<1>(mode, tm, p, st);
    case 2: return launch_step_r<2>(mode, tm, p, st);
    case 3: return launch_step_r<3>(mode, tm, p, st);
    case 4: return launch_step_r<4>(mode, tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_setup_kappa(const float *sos, const float *density, float *kap, int *status, int n_maps, int Nx,
                               int Nz, int P, int nxp, int nzp, int pitch, double dt_over_dx, double d0, double dt,
                               double c_max, cudaStream_t st)
{
    dim3 grid((pitch + 127) / 128, nzp, n_maps);
    setup_kappa_kernel<<<grid, 128, 0, st>>>(sos, density, kap, status, Nx, Nz, P, nxp, nzp, pitch,
                                             dt_over_dx * dt_over_dx, d0, dt, c_max);
    return cudaGetLastError();
}

cudaError_t launch_sample(const float *field, const int *rx_node, float *cd, long long slice, int pitch, int S,
                          int n_tx, int n_rx, int nt, int step, cudaStream_t st)
{
    if (n_rx == 0) return cudaSuccess;
    sample_kernel<<<S, 128, 0, st>>>(field, rx_node, cd, slice, pitch, n_tx, n_rx, nt, step);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float *cd_sim, const float *cd_obs, const float *kap, const int *rx_node,
                            float *asrc, double *partial, int *status, int S, int n_tx, int n_rx, int nt,
                            long long slice, int pitch, cudaStream_t st)
{
    residual_kernel<<<S, 512, 0, st>>>(cd_sim, cd_obs, kap, rx_node, asrc, partial, status, n_tx, n_rx, nt, slice,
                                       pitch);
    return cudaGetLastError();
}

cudaError_t launch_misfit_sum(const double *partial, double *misfit, int n_maps, int n_tx, cudaStream_t st)
{
    misfit_sum_kernel<<<(n_maps + 127) / 128, 128, 0, st>>>(partial, misfit, n_maps, n_tx);
    return cudaGetLastError();
}

cudaError_t launch_fold(const float *g_shot, const float *sos, float *grad, double *fx, int n_maps, int n_tx, int Nx,
                        int Nz, int P, long long slice, int pitch, cudaStream_t st)
{
    const int nzp = Nz + 2 * P;
    fold_x_kernel<<<dim3((Nx + 127) / 128, nzp, n_maps), 128, 0, st>>>(g_shot, fx, n_tx, Nx, P, nzp, slice, pitch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_z_kernel<<<dim3((Nx + 127) / 128, Nz, n_maps), 128, 0, st>>>(fx, sos, grad, Nx, Nz, P, nzp);
    return cudaGetLastError();
}

cudaError_t launch_snap_absmax(const float *cur, const float *prev, unsigned *scale_bits, int S, long long slice,
                               int, int, int, cudaStream_t st)
{
    dim3 grid(static_cast<unsigned>(std::min<long long>((slice / 4 + 255) / 256, 64)), S);
    snap_absmax_kernel<<<grid, 256, 0, st>>>(cur, prev, scale_bits, slice);
    return cudaGetLastError();
}

cudaError_t launch_snap_store(const float *cur, const float *prev, void *snap_u, void *snap_d,
                              const unsigned *scale_bits, int dtype, int S, long long slice, int, int, int,
                              cudaStream_t st)
{
    dim3 grid(static_cast<unsigned>(std::min<long long>((slice + 255) / 256, 256)), S);
    if (dtype == DUFWI_SNAP_BF16)
        snap_store_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(cur, prev, (__nv_bfloat16 *)snap_u,
                                                               (__nv_bfloat16 *)snap_d, scale_bits, dtype, slice);
    else
        snap_store_kernel<__half><<<grid, 256, 0, st>>>(cur, prev, (__half *)snap_u, (__half *)snap_d, scale_bits,
                                                        dtype, slice);
    return cudaGetLastError();
}

cudaError_t launch_snap_load(float *cur, float *prev, const void *snap_u, const void *snap_d,
                             const unsigned *scale_bits, int dtype, int S, long long slice, int, int, int,
                             cudaStream_t st)
{
    dim3 grid(static_cast<unsigned>(std::min<long long>((slice + 255) / 256, 256)), S);
    if (dtype == DUFWI_SNAP_BF16)
        snap_load_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(cur, prev, (const __nv_bfloat16 *)snap_u,
                                                              (const __nv_bfloat16 *)snap_d, scale_bits, dtype, slice);
    else
        snap_load_kernel<__half><<<grid, 256, 0, st>>>(cur, prev, (const __half *)snap_u, (const __half *)snap_d,
                                                       scale_bits, dtype, slice);
    return cudaGetLastError();
}

}  // namespace dufwi
