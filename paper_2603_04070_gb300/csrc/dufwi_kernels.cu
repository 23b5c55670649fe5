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

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/dufwi.h"
#include "dufwi_device.cuh"

namespace dufwi {

namespace {
// <one-step kernel source>

template <int MODE, int TZ>
struct TileLayout {
    static constexpr int kBoxRows = TZ + 2 * kHalo;
    static constexpr int kBox = kBoxX * kBoxRows;                      // U^n (or mu^{m+1}) with halo
    static constexpr int kTile = kTileX * TZ;
    // prev, kappa (+ history and sums in the adjoint; + Lap(U^n) and dkappa' in the Born step)
    static constexpr int kTiles = (MODE == kAdjoint || MODE == kBorn) ? 4 : 2;
    static constexpr int kFloats = kBox + kTiles * kTile;
    static constexpr uint32_t kBytes = kFloats * sizeof(float);
    static constexpr int kPasses = TZ / 32;                            // 32-row passes per CTA
    static constexpr int kThreadsPerCta = 128;                         // 4 (x) x 4 (z) outputs per pass
};

constexpr int kMaxInj = 64;   // point injections staged in shared memory per list

// Point injections of one step into a region of shared memory: source samples (forward) or
// scaled residuals at receivers (adjoint). They are gathered in parallel into shared memory
// and applied by one thread in list order, so the result is deterministic even when several
// entries hit the same node.
struct InjList {
    int n;
    int idx[kMaxInj];
    float val[kMaxInj];
};

// Fills `l` (called by every thread; a barrier must follow before use) with the injections of
// step `step` that land in the region [rz0, rz0 + rh) x [rx0, rx0 + rw) of shot s; the local
// index is (z - rz0) * stride + (x - rx0). range: (first, count) into p.rx_sorted (adjoint).
template <int MODE>
__device__ __forceinline__ void gather_injections(InjList &l, const StepParams &p, const int *sorted, int n_sorted,
                                                  int s, int tx_idx, int step, int2 range, int rx0, int rz0, int rw,
                                                  int rh, int stride, int tid, int nthreads)
{
    if (MODE == kAdjoint) {
        // Every index derived from the tables is checked before use: a damaged table raises
        // DUFWI_ERR_GEOMETRY in the status word instead of addressing outside the buffers.
        const bool range_ok = range.x >= 0 && range.y >= 0 && range.x + range.y <= n_sorted;
        if (tid == 0) {
            l.n = range_ok ? range.y : 0;
            if (!range_ok) raise_status(p.status, DUFWI_ERR_GEOMETRY);
        }
        const int m = range_ok ? min(range.y, kMaxInj) : 0;
        for (int e = tid; e < m; e += nthreads) {
            const int r = __ldg(sorted + tx_idx * n_sorted + range.x + e);
            const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.inj_node + tx_idx * p.n_rx + r) : -1;
            const int zn = node >> 16, xn = node & 0xffff;
            if (node < 0 || zn < rz0 || zn >= rz0 + rh || xn < rx0 || xn >= rx0 + rw) {
                l.idx[e] = -1;
                l.val[e] = 0.0f;
                raise_status(p.status, DUFWI_ERR_GEOMETRY);
                continue;
            }
            l.idx[e] = (zn - rz0) * stride + (xn - rx0);
            l.val[e] = __ldg(p.inj_val + (static_cast<long long>(s) * p.nt + step) * p.n_rx + r);
        }
    } else if (tid == 0) {
        const int node = __ldg(p.inj_node + tx_idx);
        const int zn = node >> 16, xn = node & 0xffff;
        const bool in = zn >= rz0 && zn < rz0 + rh && xn >= rx0 && xn < rx0 + rw;
        l.n = in ? 1 : 0;
        if (in) {
            l.idx[0] = (zn - rz0) * stride + (xn - rx0);
            l.val[0] = p.inj_scale * __ldg(p.inj_val + static_cast<long long>(p.wav_per_tx ? tx_idx : 0) * p.nt + step);
        }
    }
}

// Applies a gathered list to `buf` (thread 0 only). Entries beyond the staged capacity are read
// from global memory directly (same order).
template <int MODE>
__device__ __forceinline__ void apply_injections(const InjList &l, float *buf, const StepParams &p, const int *sorted,
                                                 int n_sorted, int s, int tx_idx, int step, int2 range, int rx0,
                                                 int rz0, int rw, int rh, int stride, int idx_lo = 0,
                                                 int idx_hi = 1 << 30)
{
    const int m = min(l.n, kMaxInj);
    for (int e = 0; e < m; ++e)
        if (l.idx[e] >= 0 && l.idx[e] >= idx_lo && l.idx[e] < idx_hi) buf[l.idx[e]] += l.val[e];
    if (MODE == kAdjoint) {
        for (int e = kMaxInj; e < l.n; ++e) {
            const int r = __ldg(sorted + tx_idx * n_sorted + range.x + e);
            const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.inj_node + tx_idx * p.n_rx + r) : -1;
            const int zn = node >> 16, xn = node & 0xffff;
            if (node < 0 || zn < rz0 || zn >= rz0 + rh || xn < rx0 || xn >= rx0 + rw) {
                raise_status(p.status, DUFWI_ERR_GEOMETRY);
                continue;
            }
            const int idx = (zn - rz0) * stride + (xn - rx0);
            if (idx >= idx_lo && idx < idx_hi)
                buf[idx] += __ldg(p.inj_val + (static_cast<long long>(s) * p.nt + step) * p.n_rx + r);
        }
    }
}

// Laplacian (difference form) of a 4 (x) x 4 (z) block of a shared-memory field with row stride
// SX whose first cell is at (cx, cz); the halo covers cx - 4 .. cx + 7 and cz - R .. cz + 3 + R.
//   lap = sum_k c_k ((x_{+k} + x_{-k}) + (z_{+k} + z_{-k}) - 4u)
// is exactly zero on a constant field whatever the rounding of the weights. The four x-lanes
// are processed as two packed FP32 pairs (f32x2 instructions, IEEE rounding and order kept).
template <int R, int SX>
__device__ __forceinline__ void lap_block(const float *src, int cx, int cz, const float *c, float4 (&lap)[4],
                                          float4 (&ctr)[4])
{
    float4 col[4 + 2 * R];
#pragma unroll
    for (int i = 0; i < 4 + 2 * R; ++i) col[i] = ld4s(src + (cz - R + i) * SX + cx);
    const float2 m4 = make_float2(-4.0f, -4.0f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 lft = ld4s(src + (cz + j) * SX + cx - 4);
        const float4 rgt = ld4s(src + (cz + j) * SX + cx + 4);
        const float4 cc = col[R + j];
        ctr[j] = cc;
        const float w[12] = {lft.x, lft.y, lft.z, lft.w, cc.x, cc.y, cc.z, cc.w, rgt.x, rgt.y, rgt.z, rgt.w};
        float2 l[2];
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
                acc = __ffma2_rn(make_float2(c[kk], c[kk]), __fadd2_rn(__fadd2_rn(xs, zs), nu4), acc);
            }
            l[h] = acc;
        }
        lap[j] = make_float4(l[0].x, l[0].y, l[1].x, l[1].y);
    }
}

// Eq. 2 for four cells of a row: 2u - p + (a - 2) u + (b + 1) p + kappa' lap. The small damping
// terms (a - 2, b + 1) come from a table over the layer depths (FP64 on the host, rounded once);
// trow is the table row of this z, xd the x depths of the four lanes.
__device__ __forceinline__ float4 eq2_row(float4 u, float4 pv, float4 kp, float4 lap, bool interior,
                                          const float2 *trow, const int (&xd)[4])
{
    const float2 two2 = make_float2(2.0f, 2.0f);
    float2 b0 = __ffma2_rn(two2, make_float2(u.x, u.y), make_float2(-pv.x, -pv.y));
    float2 b1 = __ffma2_rn(two2, make_float2(u.z, u.w), make_float2(-pv.z, -pv.w));
    if (!interior) {
        const float2 t0 = __ldg(trow + xd[0]), t1 = __ldg(trow + xd[1]);
        const float2 t2 = __ldg(trow + xd[2]), t3 = __ldg(trow + xd[3]);
        b0 = __ffma2_rn(make_float2(t0.x, t1.x), make_float2(u.x, u.y),
                        __ffma2_rn(make_float2(t0.y, t1.y), make_float2(pv.x, pv.y), b0));
        b1 = __ffma2_rn(make_float2(t2.x, t3.x), make_float2(u.z, u.w),
                        __ffma2_rn(make_float2(t2.y, t3.y), make_float2(pv.z, pv.w), b1));
    }
    const float2 n01 = __ffma2_rn(make_float2(kp.x, kp.y), make_float2(lap.x, lap.y), b0);
    const float2 n23 = __ffma2_rn(make_float2(kp.z, kp.w), make_float2(lap.z, lap.w), b1);
    return make_float4(n01.x, n01.y, n23.x, n23.y);
}

// Issues the TMA loads of one launch (thread 0) after the previous kernel in the stream is done.
__device__ __forceinline__ bool wait_tile(uint64_t *bar, const StepParams &p, int tid)
{
    int fail = 0;
    if (tid == 0) fail = !mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(fail)) {
        if (tid == 0) raise_status(p.status, DUFWI_ERR_TIMEOUT);
        mbar_wait_bounded(bar, 0);
        return false;
    }
    // every thread takes its own (immediately successful) acquire of the completed phase
    if (!mbar_try_wait_sleep(bar, 0) && !mbar_wait_bounded(bar, 0)) {
        raise_status(p.status, DUFWI_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// Minimum resident CTAs per SM requested from the register allocator. Build-time knob.
#ifndef DUFWI_STEP_MIN_CTAS_128
#define DUFWI_STEP_MIN_CTAS_128 5
#endif

// One time step, one 64 x TZ output tile of one shot per CTA (128 threads, TZ / 32 passes of
// 4 x 4 outputs per thread). A single mbarrier collects the TMA loads of the (64 + 8) x (TZ + 8)
// box of U^n and of the 64 x TZ tiles of U^{n-1} and kappa' (and, in the adjoint, of
// Lap(U^{m-1}) and of the running imaging sum). Many small CTAs stay resident per SM, so the
// loads of some overlap the arithmetic of others.
// MINB: resident CTAs per SM asked of the register allocator (0: the build default above; the
// 64 x 32 form of the 8th-order stencil is also compiled for 4 and 6, a launch option).
template <int R, int MODE, int TZ, int MINB = 0>
__global__ void __launch_bounds__(TileLayout<MODE, TZ>::kThreadsPerCta,
                                  MINB ? MINB : (TZ == 32 ? DUFWI_STEP_MIN_CTAS_128 : 4))
step_kernel(const __grid_constant__ StepMaps tm, const StepParams p)
{
    using TL = TileLayout<MODE, TZ>;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;
    __shared__ InjList inj;

    const int tid = threadIdx.x;
    const int s = p.shot0 + blockIdx.z;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * TZ;
    const int tx_idx = s % p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *box = smem;
    float *pv = box + TL::kBox;
    float *kp = pv + TL::kTile;
    float *hs = kp + TL::kTile;
    float *gg = hs + TL::kTile;
    // sized calls: tiles outside this map's padded grid have nothing to do (their cells stay zero)
    const MapGrid mg = map_grid(p, s / p.n_tx);
    if (x0 >= mg.nxp || z0 >= mg.nzp) return;

    // Thread 0 initialises the barrier, issues the loads and alone polls the barrier; the other
    // threads first touch it after the CTA barrier in wait_tile, so no barrier is needed here.
    // With p.early the operands that no launch of the last two wrote (U^{n-1}, kappa', and in the
    // adjoint the history) are requested before the wait for the previous launch, overlapping
    // its tail; the host sets it only where that holds.
    const bool early = MODE != kBorn && p.early;
    if (tid == 0) {
        prefetch_tensormap(&tm.cur_box);
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, TL::kBytes);
        if (early) {
            tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
            tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, s / p.n_tx);
            if (MODE == kAdjoint) tma_load_4d_stream(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
        }
    }
    grid_dependency_wait();
    if (tid == 0) {
        tma_load_3d(box, &tm.cur_box, &bar, x0 - kHalo, z0 - kHalo, s);
        if (!early) {
            tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
            tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, s / p.n_tx);
            if (MODE == kAdjoint) tma_load_4d_stream(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
        }
        if (MODE == kAdjoint) tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, s);
        if (MODE == kBorn) {
            tma_load_4d(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
            tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, s / p.n_tx);
        }
    }
    grid_dependents_launch();

    // Receivers of this transmit inside this tile: a host-built table gives the range of them
    // (indices into rx_sorted), so no CTA scans the whole receiver list.
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    int2 rx_range = make_int2(0, 0);
    if (MODE != kFwdHist) rx_range = __ldg(p.rx_tab + tx_idx * (gridDim.x * gridDim.y) + tile);
    if (MODE == kBorn) {   // the Born field has no point source of its own
        if (tid == 0) inj.n = 0;
    } else {
        gather_injections<MODE>(inj, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX, TZ, kTileX,
                                tid, TL::kThreadsPerCta);
    }

    const int lx = (tid & 15) * 4;
    const int gx = x0 + lx;
    const bool interior = region_interior(p, mg, x0, z0, kTileX, TZ);
    int xd[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, mg.Nx);

    if (!wait_tile(&bar, p, tid)) return;

    const bool col_ok = gx < mg.nxp;
#pragma unroll 1
    for (int pass = 0; pass < TL::kPasses; ++pass) {
        const int lz = (tid >> 4) * 4 + 32 * pass;
        float4 lap[4], ctr[4], nxt[4];
        lap_block<R, kBoxX>(box, kHalo + lx, kHalo + lz, p.c, lap, ctr);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int lo = (lz + j) * kTileX + lx;
            nxt[j] = eq2_row(ctr[j], ld4s(pv + lo), ld4s(kp + lo), lap[j], interior,
                             p.damp_tab + layer_depth(z0 + lz + j, p.P, mg.Nz) * (p.P + 1), xd);
            if (MODE == kBorn) nxt[j] = fma4(ld4s(gg + lo), ld4s(hs + lo), nxt[j]);   // + dkappa' Lap(U^n)
        }
        if (MODE != kBorn && inj.n > 0) {   // block-uniform: stage this pass's rows, inject, reload
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) st4s(pv + (lz + j) * kTileX + lx, nxt[j]);
            __syncthreads();
            if (tid == 0)
                apply_injections<MODE>(inj, pv, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX,
                                       TZ, kTileX, 32 * pass * kTileX, 32 * (pass + 1) * kTileX);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) nxt[j] = ld4s(pv + (lz + j) * kTileX + lx);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gz = z0 + lz + j;
            if (!col_ok || gz >= mg.nzp) continue;
            float4 nv = nxt[j], lv = lap[j];
            if (gx + 4 > mg.nxp) {   // lanes past the last column stay zero (outside the map's grid)
                if (gx + 1 >= mg.nxp) { nv.y = 0.f; lv.y = 0.f; }
                if (gx + 2 >= mg.nxp) { nv.z = 0.f; lv.z = 0.f; }
                nv.w = 0.f; lv.w = 0.f;
            }
            const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
            st4(p.out + o, nv);
            if (MODE == kFwdSampleHist || MODE == kFwdHist) st4_stream(p.hist + o, lv);
            if (MODE == kAdjoint) {
                const int lo = (lz + j) * kTileX + lx;
                st4(p.grad + o, fma4(nv, ld4s(hs + lo), ld4s(gg + lo)));
            }
        }
    }

    // Receiver sampling of U^n from the box (each receiver lies in exactly one tile).
    if (MODE == kFwdSample || MODE == kFwdSampleHist || MODE == kBorn) {
        const int cnt = (rx_range.x >= 0 && rx_range.y >= 0 && rx_range.x + rx_range.y <= p.n_rx) ? rx_range.y : 0;
        for (int e = tid; e < cnt; e += TL::kThreadsPerCta) {
            const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
            const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
            const int zn = node >> 16, xn = node & 0xffff;
            if (node < 0 || zn < z0 || zn >= z0 + TZ || xn < x0 || xn >= x0 + kTileX) {
                raise_status(p.status, DUFWI_ERR_GEOMETRY);
                continue;
            }
            p.cd[(static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r] =
                box[(zn - z0 + kHalo) * kBoxX + (xn - x0 + kHalo)];
        }
    }
}

// Multi-tile form of the one-step kernel. A grid of G CTAs (as many as fit on the device at
// once) walks the 64 x 32 tiles of all shots: CTA b takes tiles t = b, b + G, b + 2G, ... (t runs
// over shots, then tile rows, then tile columns). Two shared-memory stages, each with its own
// mbarrier, hold the operands of two tiles: the TMA loads of tile i + 1 are issued before tile i
// is computed, so their latency overlaps the arithmetic instead of being exposed once per CTA as
// in the one-tile-per-CTA form, and the tiles are spread evenly over the CTAs (no partial last
// wave). The arithmetic, injections, sampling and stores per tile are those of step_kernel with
// TZ = 32, so the results are bit-identical.
template <int R, int MODE>
__global__ void __launch_bounds__(128, (MODE == kAdjoint || MODE == kBorn) ? 2 : 4)
step_mt_kernel(const __grid_constant__ StepMaps tm, const StepParams p)
{
    using TL = TileLayout<MODE, 32>;
    constexpr int TZ = 32;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar[2];
    __shared__ InjList inj;

    const int tid = threadIdx.x;
    const int tiles_x = (p.nxp + kTileX - 1) / kTileX;
    const int per_shot = tiles_x * ((p.nzp + TZ - 1) / TZ);
    const int total = p.n_maps * p.n_tx * per_shot;
    const int G = gridDim.x;
    const bool early = MODE != kBorn && p.early;

    // tile t -> shot, origin and row-major tile index within the shot; false for tiles outside the
    // shot's own grid (sized calls), which have nothing to do
    auto locate = [&](int t, int &s, int &x0, int &z0, int &tile) {
        s = t / per_shot;
        tile = t - s * per_shot;
        x0 = (tile % tiles_x) * kTileX;
        z0 = (tile / tiles_x) * TZ;
        const MapGrid g = map_grid(p, s / p.n_tx);
        return x0 < g.nxp && z0 < g.nzp;
    };
    auto stage_base = [&](int k) { return smem + k * TL::kFloats; };
    // thread 0: the loads of tile t into stage k (part 1: operands no launch of the last two wrote;
    // part 2: the box of U^n and, in the adjoint, the imaging sums)
    auto issue = [&](int t, int k, bool part1, bool part2) {
        int s, x0, z0, tile;
        locate(t, s, x0, z0, tile);
        float *box = stage_base(k), *pv = box + TL::kBox, *kp = pv + TL::kTile, *hs = kp + TL::kTile;
        float *gg = hs + TL::kTile;
        if (part1) {
            tma_load_3d(pv, &tm.out_tile, &bar[k], x0, z0, s);
            tma_load_3d(kp, &tm.kap_tile, &bar[k], x0, z0, s / p.n_tx);
            if (MODE == kAdjoint) tma_load_4d_stream(hs, &tm.hist_tile, &bar[k], x0, z0, s, p.hist_slot);
            if (MODE == kBorn) {
                tma_load_4d(hs, &tm.hist_tile, &bar[k], x0, z0, s, p.hist_slot);
                tma_load_3d(gg, &tm.grad_tile, &bar[k], x0, z0, s / p.n_tx);
            }
        }
        if (part2) {
            tma_load_3d(box, &tm.cur_box, &bar[k], x0 - kHalo, z0 - kHalo, s);
            if (MODE == kAdjoint) tma_load_3d(gg, &tm.grad_tile, &bar[k], x0, z0, s);
        }
    };

    if (tid == 0) {
        prefetch_tensormap(&tm.cur_box);
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();   // barriers initialised before any thread polls them
    int s0, x00, z00, tile0;
    const bool first_valid = blockIdx.x < total && locate(blockIdx.x, s0, x00, z00, tile0);
    if (tid == 0 && first_valid) {
        mbar_arrive_expect_tx(&bar[0], TL::kBytes);
        if (early) issue(blockIdx.x, 0, true, false);
    }
    grid_dependency_wait();
    if (tid == 0 && first_valid) issue(blockIdx.x, 0, !early, true);
    grid_dependents_launch();

    uint32_t parity = 0;   // bit k: phase parity of the next completion of stage k
    const int lx = (tid & 15) * 4;
    const int lz = (tid >> 4) * 4;
    int i = 0;
    for (int t = blockIdx.x; t < total; t += G, ++i) {
        const int k = i & 1;
        // the loads of the next tile go to the other stage, which the previous iteration released
        const int tn = t + G;
        int sn, xn, zn, tilen;
        const bool next_valid = tn < total && locate(tn, sn, xn, zn, tilen);
        if (tid == 0 && next_valid) {
            fence_proxy_async_shared();
            mbar_arrive_expect_tx(&bar[k ^ 1], TL::kBytes);
            issue(tn, k ^ 1, true, true);
        }
        int s, x0, z0, tile;
        if (!locate(t, s, x0, z0, tile)) {
            __syncthreads();
            continue;
        }
        const int tx_idx = s % p.n_tx;
        const long long shot_off = static_cast<long long>(s) * p.slice;
        const MapGrid mg = map_grid(p, s / p.n_tx);
        float *box = stage_base(k), *pv = box + TL::kBox, *kp = pv + TL::kTile, *hs = kp + TL::kTile;
        float *gg = hs + TL::kTile;

        int2 rx_range = make_int2(0, 0);
        if (MODE != kFwdHist) rx_range = __ldg(p.rx_tab + tx_idx * per_shot + tile);
        if (MODE == kBorn) {
            if (tid == 0) inj.n = 0;
        } else {
            gather_injections<MODE>(inj, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX, TZ,
                                    kTileX, tid, TL::kThreadsPerCta);
        }
        const int gx = x0 + lx;
        const bool interior = region_interior(p, mg, x0, z0, kTileX, TZ);
        int xd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) xd[q] = layer_depth(gx + q, p.P, mg.Nx);

        const uint32_t pk = (parity >> k) & 1u;
        const int fail = !mbar_wait_bounded(&bar[k], pk);
        if (__syncthreads_or(fail)) {   // also publishes the injection list
            if (tid == 0) raise_status(p.status, DUFWI_ERR_TIMEOUT);
            mbar_wait_bounded(&bar[k], pk);                                        // copies still in flight
            if (next_valid) mbar_wait_bounded(&bar[k ^ 1], (parity >> (k ^ 1)) & 1u);
            return;
        }
        parity ^= 1u << k;

        const bool col_ok = gx < mg.nxp;
        float4 lap[4], ctr[4], nxt[4];
        lap_block<R, kBoxX>(box, kHalo + lx, kHalo + lz, p.c, lap, ctr);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int lo = (lz + j) * kTileX + lx;
            nxt[j] = eq2_row(ctr[j], ld4s(pv + lo), ld4s(kp + lo), lap[j], interior,
                             p.damp_tab + layer_depth(z0 + lz + j, p.P, mg.Nz) * (p.P + 1), xd);
            if (MODE == kBorn) nxt[j] = fma4(ld4s(gg + lo), ld4s(hs + lo), nxt[j]);
        }
        if (MODE != kBorn && inj.n > 0) {   // block-uniform: stage the rows, inject, reload
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) st4s(pv + (lz + j) * kTileX + lx, nxt[j]);
            __syncthreads();
            if (tid == 0)
                apply_injections<MODE>(inj, pv, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX,
                                       TZ, kTileX, 0, TZ * kTileX);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) nxt[j] = ld4s(pv + (lz + j) * kTileX + lx);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gz = z0 + lz + j;
            if (!col_ok || gz >= mg.nzp) continue;
            float4 nv = nxt[j], lv = lap[j];
            if (gx + 4 > mg.nxp) {
                if (gx + 1 >= mg.nxp) { nv.y = 0.f; lv.y = 0.f; }
                if (gx + 2 >= mg.nxp) { nv.z = 0.f; lv.z = 0.f; }
                nv.w = 0.f; lv.w = 0.f;
            }
            const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
            st4(p.out + o, nv);
            if (MODE == kFwdSampleHist || MODE == kFwdHist) st4_stream(p.hist + o, lv);
            if (MODE == kAdjoint) {
                const int lo = (lz + j) * kTileX + lx;
                st4(p.grad + o, fma4(nv, ld4s(hs + lo), ld4s(gg + lo)));
            }
        }
        if (MODE == kFwdSample || MODE == kFwdSampleHist || MODE == kBorn) {
            const int cnt = (rx_range.x >= 0 && rx_range.y >= 0 && rx_range.x + rx_range.y <= p.n_rx) ? rx_range.y : 0;
            for (int e = tid; e < cnt; e += TL::kThreadsPerCta) {
                const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
                const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
                const int zn2 = node >> 16, xn2 = node & 0xffff;
                if (node < 0 || zn2 < z0 || zn2 >= z0 + TZ || xn2 < x0 || xn2 >= x0 + kTileX) {
                    raise_status(p.status, DUFWI_ERR_GEOMETRY);
                    continue;
                }
                p.cd[(static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r] =
                    box[(zn2 - z0 + kHalo) * kBoxX + (xn2 - x0 + kHalo)];
            }
        }
        __syncthreads();   // stage k and the injection list are free for reuse
    }
}

// </one-step kernel source>

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// The staggered operator of Eq. 1, G = D-_x(b_x D+_x u) + D-_z(b_z D+_z u) (unscaled), at the 4 x 4
// block of cells (lx .. lx + 3, lz .. lz + 3) of a 64 x 32 tile: box is the 80 x 48 field box (column
// 0 = x0 - 8, row 0 = z0 - 8), bxs the 72 x 32 x-buoyancy tile (column h = half point
// x0 - 4 + h + 1/2), bzs the 64 x 40 z-buoyancy tile (row j = half point z0 - 4 + j + 1/2), sw the
// staggered weights. lap receives G, ctr the field at the block's cells.
// z-fluxes of a whole 64 x 32 tile, each formed once: F[r] = b_z[r] sum_k s_k (box[r + 4 + k] -
// box[r + 5 - k]) at the half-point rows r = 0 .. 38 of the z-buoyancy tile (box row 0 is z0 - 8),
// for the 16 column quads, written over the buoyancy tile (each element is read and then written
// by the same thread). Thread (quad tid & 15, group tid >> 4) takes rows 5g .. 5g + 4 from a
// window of 12 box rows. Each flux is the same operations, in the same order, as in the register
// form of vd_operator_block, so the two forms give identical results.
template <int R>
__device__ __forceinline__ void vd_zflux_tile(const float *box, float *bzs, const float *sw, int tid)
{
    const int lx = (tid & 15) * 4;
    const int r0 = 5 * (tid >> 4);
    float4 col[12];   // box rows r0 + 1 .. r0 + 12
#pragma unroll
    for (int i = 0; i < 12; ++i) col[i] = ld4s(box + (r0 + 1 + i) * kVBoxX + lx + kVHalo);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const int r = r0 + f;
        if (r > 38) break;   // the last group's fifth row is not read
        float2 d[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            const float4 up = col[f + 3 + k], dn = col[f + 4 - k];
            const float2 sk = make_float2(sw[k - 1], sw[k - 1]);
            d[0] = __ffma2_rn(sk, __fadd2_rn(make_float2(up.x, up.y), neg2(make_float2(dn.x, dn.y))), d[0]);
            d[1] = __ffma2_rn(sk, __fadd2_rn(make_float2(up.z, up.w), neg2(make_float2(dn.z, dn.w))), d[1]);
        }
        float *bp = bzs + r * kTileX + lx;
        const float4 b = ld4s(bp);
        const float2 f0 = __fmul2_rn(make_float2(b.x, b.y), d[0]), f1 = __fmul2_rn(make_float2(b.z, b.w), d[1]);
        st4s(bp, make_float4(f0.x, f0.y, f1.x, f1.y));
    }
}

// ZF: bzs holds the z-fluxes of the tile (vd_zflux_tile) instead of the z-buoyancies.
template <int R, bool ZF = false>
__device__ __forceinline__ void vd_operator_block(const float *box, const float *bxs, const float *bzs, int lx, int lz,
                                                  const float *sw, float4 (&lap)[4], float4 (&ctr)[4])
{
    // The arithmetic runs on packed FP32 pairs (f32x2: the same IEEE operations per lane, in the
    // same order as the scalar form). Along x the pairs are two neighbouring half points (fluxes)
    // or two neighbouring cells (divergence), built once per row from shifted copies so that
    // every packed operand is an aligned register pair; along z they are two columns of a float4.
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float *row = box + (lz + j + kVHalo) * kVBoxX + lx;
        float w[20];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float4 v = ld4s(row + 4 * c);
            w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
        }
        const float *brow = bxs + (lz + j) * kVFxX + lx;
        float bw[12];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 v = ld4s(brow + 4 * c);
            bw[4 * c] = v.x; bw[4 * c + 1] = v.y; bw[4 * c + 2] = v.z; bw[4 * c + 3] = v.w;
        }
        // flux h (h = 0..10) = bw[h] sum_k s_k (w[h + 4 + k] - w[h + 5 - k]); pairs (h, h + 1), h even
        float flux[12];
#pragma unroll
        for (int h = 0; h < 12; h += 2) {
            float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                const float2 hi = make_float2(w[h + 4 + k], h + 5 + k < 20 ? w[h + 5 + k] : 0.0f);
                const float2 lo = make_float2(w[h + 5 - k], w[h + 6 - k]);
                acc = __ffma2_rn(make_float2(sw[k - 1], sw[k - 1]), __fadd2_rn(hi, neg2(lo)), acc);
            }
            const float2 f = __fmul2_rn(make_float2(bw[h], bw[h + 1]), acc);
            flux[h] = f.x;
            flux[h + 1] = f.y;
        }
        // divergence at cells q = 0..3: sum_k s_k (flux[q + k + 3] - flux[q - k + 4]); pairs (q, q + 1)
        float2 lxv[2];
#pragma unroll
        for (int q = 0; q < 4; q += 2) {
            float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 1; k <= R; ++k)
                acc = __ffma2_rn(make_float2(sw[k - 1], sw[k - 1]),
                                 __fadd2_rn(make_float2(flux[q + k + 3], flux[q + k + 4]),
                                            neg2(make_float2(flux[q - k + 4], flux[q - k + 5]))),
                                 acc);
            lxv[q / 2] = acc;
        }
        lap[j] = make_float4(lxv[0].x, lxv[0].y, lxv[1].x, lxv[1].y);
        ctr[j] = make_float4(w[8], w[9], w[10], w[11]);
    }
    if (ZF) {   // the tile's z-fluxes are in shared memory: divergence only
        float2 lzv[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) lzv[j][0] = lzv[j][1] = make_float2(0.f, 0.f);
#pragma unroll
        for (int f = 0; f < 11; ++f) {
            const float4 F = ld4s(bzs + (lz + f) * kTileX + lx);
            const float2 fl[2] = {make_float2(F.x, F.y), make_float2(F.z, F.w)};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kp_ = f - j - 3, km_ = j + 4 - f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (kp_ >= 1 && kp_ <= R)
                        lzv[j][h] = __ffma2_rn(make_float2(sw[kp_ - 1], sw[kp_ - 1]), fl[h], lzv[j][h]);
                    if (km_ >= 1 && km_ <= R)
                        lzv[j][h] = __ffma2_rn(make_float2(-sw[km_ - 1], -sw[km_ - 1]), fl[h], lzv[j][h]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 a01 = __fadd2_rn(make_float2(lap[j].x, lap[j].y), lzv[j][0]);
            const float2 a23 = __fadd2_rn(make_float2(lap[j].z, lap[j].w), lzv[j][1]);
            lap[j] = make_float4(a01.x, a01.y, a23.x, a23.y);
        }
    } else {
        float4 col[18];
#pragma unroll
        for (int r = 0; r < 18; ++r) col[r] = ld4s(box + (lz + 1 + r) * kVBoxX + lx + kVHalo);
        float2 lzv[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) lzv[j][0] = lzv[j][1] = make_float2(0.f, 0.f);
#pragma unroll
        for (int f = 0; f < 11; ++f) {
            // flux at half-point row lz + f: box rows lz + f + 4 + k and lz + f + 5 - k = col[f + 3 + k], col[f + 4 - k]
            float2 d[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                const float4 up = col[f + 3 + k], dn = col[f + 4 - k];
                const float2 sk = make_float2(sw[k - 1], sw[k - 1]);
                d[0] = __ffma2_rn(sk, __fadd2_rn(make_float2(up.x, up.y), neg2(make_float2(dn.x, dn.y))), d[0]);
                d[1] = __ffma2_rn(sk, __fadd2_rn(make_float2(up.z, up.w), neg2(make_float2(dn.z, dn.w))), d[1]);
            }
            const float4 b = ld4s(bzs + (lz + f) * kTileX + lx);
            const float2 fl[2] = {__fmul2_rn(make_float2(b.x, b.y), d[0]), __fmul2_rn(make_float2(b.z, b.w), d[1])};
            // output row j takes +s_k from flux j + k + 3 and -s_k from flux j - k + 4
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kp_ = f - j - 3, km_ = j + 4 - f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (kp_ >= 1 && kp_ <= R)
                        lzv[j][h] = __ffma2_rn(make_float2(sw[kp_ - 1], sw[kp_ - 1]), fl[h], lzv[j][h]);
                    if (km_ >= 1 && km_ <= R)
                        lzv[j][h] = __ffma2_rn(make_float2(-sw[km_ - 1], -sw[km_ - 1]), fl[h], lzv[j][h]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 a01 = __fadd2_rn(make_float2(lap[j].x, lap[j].y), lzv[j][0]);
            const float2 a23 = __fadd2_rn(make_float2(lap[j].z, lap[j].w), lzv[j][1]);
            lap[j] = make_float4(a01.x, a01.y, a23.x, a23.y);
        }
    }
}

// CPML split: does the 64 x 32 tile at (x0, z0), grown by 8 cells, lie inside the physical grid
// (where every CPML coefficient is the identity, so that the memory variables stay zero)?
__device__ __forceinline__ bool cpml_free_tile(const StepParams &p, int x0, int z0)
{
    return x0 - 2 * kHalo >= p.P && x0 + kTileX + 2 * kHalo <= p.P + p.Nx - 1 && z0 - 2 * kHalo >= p.P &&
           z0 + kVTileZ + 2 * kHalo <= p.P + p.Nz - 1;
}

// ---- second-order products ---------------------------------------------------------------------
// For a cotangent w on the channel data and an SoS direction v, the derivative along v of
// G = (dM/dC)^T w (Eq. 6 for w = 2 (M - M_obs)) follows from differentiating the discrete adjoint
// once more. With dkappa' = 2 kappa' v / C:
//   dU^{n+1} = Eq. 2 on dU + dkappa' Lap(U^n)                         (Born field)
//   mu^m     = Eq. 2 on mu + kappa' w^m at the receivers              (adjoint, mu = kappa' lambda)
//   dmu^m    = Eq. 2 on dmu + dkappa' Lap(mu^{m+1}) + dkappa' w^m     (derivative of mu along v)
//   dG = (2/C) sum_m [dmu^m Lap(U^{m-1}) + mu^m Lap(dU^{m-1})] - (2 v / C^2) sum_m mu^m Lap(U^{m-1})
// so_step_kernel advances one of the three fields by one step with the extra terms of its kind
// (SoKind). It is the one-step kernel's tile scheme (64 x 32 tiles, 128 threads, 4 x 4 outputs
// per thread, one mbarrier for all TMA loads) with more operand tiles and no early loads.
template <int KIND, bool VD>
struct SoLayout {
    // the field box: 72 x 40 (halo 4) for the compact Laplacian, 80 x 48 (halo 8) and the two
    // half-point buoyancy tiles (72 x 32, 64 x 40) for the staggered variable-density operator
    static constexpr int kBox = VD ? kVBoxX * kVBoxZ : kBoxX * (32 + 2 * kHalo);
    static constexpr int kB = VD ? kVFxX * kVTileZ + kTileX * kVFzZ : 0;
    static constexpr int kTile = kTileX * 32;
    // prev, kappa' + (Born: Lap(U^n), dkappa'; adjoint: two histories, two sums;
    // Born-adjoint: history, Lap(mu^{m+1}), dkappa', sum)
    static constexpr int kTiles = KIND == kSoBorn ? 4 : 6;
    static constexpr uint32_t kBytes = (kBox + kB + kTiles * kTile) * sizeof(float);
};

template <int R, int KIND, bool VD>
__global__ void __launch_bounds__(128, VD ? 2 : 3)
so_step_kernel(const __grid_constant__ SoMaps tm, const StepParams p, const SoParams q)
{
    using SL = SoLayout<KIND, VD>;
    constexpr int kH = VD ? kVHalo : kHalo;        // halo of the field box
    constexpr int kSX = VD ? kVBoxX : kBoxX;       // its row stride
    constexpr int TZ = 32;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;
    __shared__ InjList inj;

    const int tid = threadIdx.x;
    const int s = p.shot0 + blockIdx.z;
    const int map = s / p.n_tx;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * TZ;
    const int tx_idx = s % p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *box = smem;
    float *fxb = box + SL::kBox;                   // buoyancy tiles (variable density)
    float *fzb = fxb + (VD ? kVFxX * kVTileZ : 0);
    float *pv = box + SL::kBox + SL::kB;
    float *kp = pv + SL::kTile;
    float *t0 = kp + SL::kTile;
    float *t1 = t0 + SL::kTile;
    float *t2 = t1 + SL::kTile;
    float *t3 = t2 + SL::kTile;
    const MapGrid mg = map_grid(p, map);
    if (VD && p.tile_class == 1 && !cpml_free_tile(p, x0, z0)) return;   // CPML: layer tiles run elsewhere

    if (tid == 0) {
        prefetch_tensormap(&tm.cur_box);
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, SL::kBytes);
    }
    grid_dependency_wait();
    if (tid == 0) {
        tma_load_3d(box, &tm.cur_box, &bar, x0 - kH, z0 - kH, s);
        if (VD) {
            tma_load_3d(fxb, &tm.bx, &bar, x0 - kHalo, z0, map);
            tma_load_3d(fzb, &tm.bz, &bar, x0, z0 - kHalo, map);
        }
        tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
        tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, map);
        tma_load_4d(t0, &tm.h1, &bar, x0, z0, s, q.h1_slot);
        if (KIND == kSoBorn) {
            tma_load_3d(t1, &tm.dk, &bar, x0, z0, map);
        } else if (KIND == kSoAdj) {
            tma_load_4d(t1, &tm.h2, &bar, x0, z0, s, q.h2_slot);
            tma_load_3d(t2, &tm.g1, &bar, x0, z0, s);
            tma_load_3d(t3, &tm.g2, &bar, x0, z0, s);
        } else {
            tma_load_3d(t1, &tm.src, &bar, x0, z0, s);
            tma_load_3d(t2, &tm.dk, &bar, x0, z0, map);
            tma_load_3d(t3, &tm.g1, &bar, x0, z0, s);
        }
    }
    grid_dependents_launch();

    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int2 rx_range = __ldg(p.rx_tab + tx_idx * (gridDim.x * gridDim.y) + tile);
    if (KIND == kSoBorn) {   // the Born field has no point source of its own
        if (tid == 0) inj.n = 0;
    } else {                 // kappa' w (adjoint) or dkappa' w (Born-adjoint) at the receivers
        gather_injections<kAdjoint>(inj, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX, TZ,
                                    kTileX, tid, 128);
    }

    const int lx = (tid & 15) * 4;
    const int gx = x0 + lx;
    const int lz = (tid >> 4) * 4;
    const bool interior = region_interior(p, mg, x0, z0, kTileX, TZ);
    int xd[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, mg.Nx);

    if (!wait_tile(&bar, p, tid)) return;

    float4 lap[4], ctr[4], nxt[4];
    if (VD)
        vd_operator_block<R>(box, fxb, fzb, lx, lz, p.sw, lap, ctr);
    else
        lap_block<R, kBoxX>(box, kHalo + lx, kHalo + lz, p.c, lap, ctr);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int lo = (lz + j) * kTileX + lx;
        nxt[j] = eq2_row(ctr[j], ld4s(pv + lo), ld4s(kp + lo), lap[j], interior,
                         p.damp_tab + layer_depth(z0 + lz + j, p.P, mg.Nz) * (p.P + 1), xd);
        if (KIND == kSoBorn) nxt[j] = fma4(ld4s(t1 + lo), ld4s(t0 + lo), nxt[j]);      // + dkappa' Lap(U^n)
        if (KIND == kSoBornAdj) nxt[j] = fma4(ld4s(t2 + lo), ld4s(t1 + lo), nxt[j]);   // + dkappa' Lap(mu^{m+1})
    }
    if (KIND != kSoBorn && inj.n > 0) {   // block-uniform: stage the rows, inject, reload
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) st4s(pv + (lz + j) * kTileX + lx, nxt[j]);
        __syncthreads();
        if (tid == 0)
            apply_injections<kAdjoint>(inj, pv, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX,
                                       TZ, kTileX);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) nxt[j] = ld4s(pv + (lz + j) * kTileX + lx);
    }
    const bool col_ok = gx < mg.nxp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gz = z0 + lz + j;
        if (!col_ok || gz >= mg.nzp) continue;
        float4 nv = nxt[j], lv = lap[j];
        if (gx + 4 > mg.nxp) {   // lanes past the last column stay zero
            if (gx + 1 >= mg.nxp) { nv.y = 0.f; lv.y = 0.f; }
            if (gx + 2 >= mg.nxp) { nv.z = 0.f; lv.z = 0.f; }
            nv.w = 0.f; lv.w = 0.f;
        }
        const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
        const int lo = (lz + j) * kTileX + lx;
        st4(p.out + o, nv);
        if (KIND == kSoBorn || KIND == kSoAdj) st4(q.lap_out + o, lv);
        if (KIND == kSoAdj) {
            st4(q.sum1 + o, fma4(nv, ld4s(t0 + lo), ld4s(t2 + lo)));
            st4(q.sum2 + o, fma4(nv, ld4s(t1 + lo), ld4s(t3 + lo)));
        }
        if (KIND == kSoBornAdj) st4(q.sum1 + o, fma4(nv, ld4s(t0 + lo), ld4s(t3 + lo)));
    }

    // Born traces: dU^n at the receivers, from the box (each receiver lies in exactly one tile)
    if (KIND == kSoBorn && p.cd) {
        const int cnt = (rx_range.x >= 0 && rx_range.y >= 0 && rx_range.x + rx_range.y <= p.n_rx) ? rx_range.y : 0;
        for (int e = tid; e < cnt; e += 128) {
            const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
            const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
            const int zn = node >> 16, xn = node & 0xffff;
            if (node < 0 || zn < z0 || zn >= z0 + TZ || xn < x0 || xn >= x0 + kTileX) {
                raise_status(p.status, DUFWI_ERR_GEOMETRY);
                continue;
            }
            p.cd[(static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r] =
                box[(zn - z0 + kH) * kSX + (xn - x0 + kH)];
        }
    }
}

// Receiver source of the differentiated adjoint for the exact Hessian-vector product of the
// misfit: dkappa'_r w + kappa'_r 2 (J v) with w = 2 (M - M_obs). The adjoint of 2 J v obeys the
// same recursion as dmu, so it rides on dmu's source and the two share one imaging sum.
__global__ void hvp_source_kernel(const float *cd_sim, const float *cd_obs, const float *dcd, const float *kap,
                                  const float *dkap, const int *rx_node, float *asrc2, int n_tx, int n_rx, int nt,
                                  long long slice, int pitch)
{
    const int s = blockIdx.y;
    const int tx_idx = s % n_tx, map = s / n_tx;
    const long long base = static_cast<long long>(s) * nt * n_rx;
    const long long n = static_cast<long long>(nt) * n_rx;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(i % n_rx);
        const int node = rx_node[tx_idx * n_rx + r];
        const long long o = map * slice + static_cast<long long>(node >> 16) * pitch + (node & 0xffff);
        const float w = 2.0f * (cd_sim[base + i] - cd_obs[base + i]);
        asrc2[base + i] = dkap[o] * w + kap[o] * (2.0f * dcd[base + i]);
    }
}

// a += b - (v / C) g per padded cell of every shot (v, C edge-replicated), before the fold.
__global__ void so_combine_kernel(float *a, const float *b, const float *g, const float *sos, const float *dsos,
                                  int n_tx, int Nx, int Nz, int P, int pitch, long long slice)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int s = blockIdx.z;
    if (x >= pitch) return;
    const int map = s / n_tx;
    const int xs = min(max(x - P, 0), Nx - 1), zs = min(max(z - P, 0), Nz - 1);
    const long long src = (static_cast<long long>(map) * Nz + zs) * Nx + xs;
    const float r = dsos[src] / sos[src];
    const long long o = static_cast<long long>(s) * slice + static_cast<long long>(z) * pitch + x;
    a[o] = (a[o] + b[o]) - r * g[o];
}

// ---- variable density (Eq. 1 with rho(x, z)) ---------------------------------------------------
// The density term rho div(b grad u), b = 1/rho, on a staggered grid. Fluxes at half points,
//   f_x(j + 1/2) = b_x(j) sum_k s_k (u(j + k) - u(j - k + 1)),
// and their divergence at the nodes, L u(x) = sum_k s_k (f_x(x + k - 1/2) - f_x(x - k + 1/2)) + the
// same along z; kappa' carries rho and 1/dx^2. With u = 0 and b = 0 outside the padded grid
// (the TMA zero fill, and b = 0 stored past the last node), L = -G^T B G is symmetric, so the
// adjoint in mu = kappa' lambda form is again the forward update, and the imaging term is
// mu^m L U^{m-1} as for the compact Laplacian.
//
// One CTA: a 64 x 32 output tile of one shot, 128 threads. TMA brings the 80 x 48 box of U^n and
// the 72 x 32 and 64 x 40 tiles of half-point buoyancies (plus U^{n-1}, kappa' and, in the
// adjoint, the history and the imaging sums) onto one mbarrier. Each thread then forms, in
// registers, the x fluxes of its four rows and the z fluxes of its four columns that its 4 x 4
// block needs (11 half points each way, shared-memory reads of 128 bits), their divergence, and
// runs the common Eq. 2 epilogue.
template <int MODE>
struct VdLayout {
    static constexpr int kBox = kVBoxX * kVBoxZ;
    static constexpr int kFx = kVFxX * kVTileZ;
    static constexpr int kFz = kTileX * kVFzZ;
    static constexpr int kTile = kTileX * kVTileZ;
    // prev, kappa' (+ history and sums in the adjoint; + Lap(U^n) and dkappa' in the Born step)
    static constexpr int kTiles = (MODE == kAdjoint || MODE == kBorn) ? 4 : 2;
    static constexpr int kFloats = kBox + kFx + kFz + kTiles * kTile;
    static constexpr uint32_t kBytes = kFloats * sizeof(float);
};

template <int R, int MODE>
__global__ void __launch_bounds__(128, 4) vd_step_kernel(const __grid_constant__ StepMaps tm, const StepParams p)
{
    using VL = VdLayout<MODE>;
    constexpr int TZ = kVTileZ;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;
    __shared__ InjList inj;

    const int tid = threadIdx.x;
    const int s = p.shot0 + blockIdx.z;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * TZ;
    const int tx_idx = s % p.n_tx;
    const int map = s / p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *box = smem;
    float *fx = box + VL::kBox;
    float *fz = fx + VL::kFx;
    float *pv = fz + VL::kFz;
    float *kp = pv + VL::kTile;
    float *hs = kp + VL::kTile;
    float *gg = hs + VL::kTile;
    const MapGrid mg = map_grid(p, map);
    if (x0 >= mg.nxp || z0 >= mg.nzp) return;
    if (p.tile_class == 1 && !cpml_free_tile(p, x0, z0)) return;   // CPML split: layer tiles run elsewhere

    // operands that neither of the last two launches wrote may be requested before the wait
    // (p.early, as in the one-step kernel)
    if (tid == 0) {
        prefetch_tensormap(&tm.cur_box);
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, VL::kBytes);
        if (MODE != kBorn && p.early) {
            tma_load_3d(fx, &tm.bx_tile, &bar, x0 - kHalo, z0, map);
            tma_load_3d(fz, &tm.bz_tile, &bar, x0, z0 - kHalo, map);
            tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
            tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, map);
            if (MODE == kAdjoint) tma_load_4d_stream(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
        }
    }
    grid_dependency_wait();
    if (tid == 0) {
        tma_load_3d(box, &tm.cur_box, &bar, x0 - kVHalo, z0 - kVHalo, s);
        if (MODE == kBorn || !p.early) {
            tma_load_3d(fx, &tm.bx_tile, &bar, x0 - kHalo, z0, map);
            tma_load_3d(fz, &tm.bz_tile, &bar, x0, z0 - kHalo, map);
            tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
            tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, map);
            if (MODE == kAdjoint) tma_load_4d_stream(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
        }
        if (MODE == kAdjoint) tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, s);
        if (MODE == kBorn) {   // Lap(U^n) of the background step, dkappa'
            tma_load_4d(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
            tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, map);
        }
    }
    grid_dependents_launch();

    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    int2 rx_range = make_int2(0, 0);
    if (MODE != kFwdHist) rx_range = __ldg(p.rx_tab + tx_idx * (gridDim.x * gridDim.y) + tile);
    if (MODE == kBorn) {   // the Born field has no point source of its own
        if (tid == 0) inj.n = 0;
    } else {
        gather_injections<MODE>(inj, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX, TZ, kTileX,
                                tid, 128);
    }

    const int lx = (tid & 15) * 4;
    const int lz = (tid >> 4) * 4;
    const int gx = x0 + lx;
    const bool interior = region_interior(p, mg, x0, z0, kTileX, TZ);
    int xd[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, mg.Nx);

    if (!wait_tile(&bar, p, tid)) return;

    // Each thread forms the fluxes its 4 x 4 block needs in registers: along x, the half points
    // lx .. lx + 10 of each of its rows (box columns lx + 1 .. lx + 18, buoyancy tile columns
    // lx .. lx + 10); along z, the half-point rows lz .. lz + 10 of its four columns (box rows
    // lz + 1 .. lz + 18, buoyancy tile rows lz .. lz + 10). Box column/row 0 is x0 - 8 / z0 - 8;
    // x-buoyancy column h is the half point x0 - 4 + h + 1/2, z-buoyancy row j is z0 - 4 + j + 1/2.
    // The z-fluxes are formed once per tile into shared memory (over the z-buoyancy tile), the
    // x-fluxes per block in registers.
    float4 lap[4], ctr[4], nxt[4];
    vd_zflux_tile<R>(box, fz, p.sw, tid);
    __syncthreads();
    vd_operator_block<R, true>(box, fx, fz, lx, lz, p.sw, lap, ctr);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int lo = (lz + j) * kTileX + lx;
        nxt[j] = eq2_row(ctr[j], ld4s(pv + lo), ld4s(kp + lo), lap[j], interior,
                         p.damp_tab + layer_depth(z0 + lz + j, p.P, mg.Nz) * (p.P + 1), xd);
        if (MODE == kBorn) nxt[j] = fma4(ld4s(gg + lo), ld4s(hs + lo), nxt[j]);   // + dkappa' L(U^n)
    }
    if (MODE != kBorn && inj.n > 0) {   // block-uniform: stage the rows, inject in list order, reload
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) st4s(pv + (lz + j) * kTileX + lx, nxt[j]);
        __syncthreads();
        if (tid == 0)
            apply_injections<MODE>(inj, pv, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX, TZ,
                                   kTileX);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) nxt[j] = ld4s(pv + (lz + j) * kTileX + lx);
    }
    const bool col_ok = gx < mg.nxp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gz = z0 + lz + j;
        if (!col_ok || gz >= mg.nzp) continue;
        float4 nv = nxt[j], lv = lap[j];
        if (gx + 4 > mg.nxp) {
            if (gx + 1 >= mg.nxp) { nv.y = 0.f; lv.y = 0.f; }
            if (gx + 2 >= mg.nxp) { nv.z = 0.f; lv.z = 0.f; }
            nv.w = 0.f; lv.w = 0.f;
        }
        const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
        st4(p.out + o, nv);
        if (MODE == kFwdSampleHist || MODE == kFwdHist) st4_stream(p.hist + o, lv);
        if (MODE == kAdjoint) {
            const int lo = (lz + j) * kTileX + lx;
            st4(p.grad + o, fma4(nv, ld4s(hs + lo), ld4s(gg + lo)));
        }
    }

    if (MODE == kFwdSample || MODE == kFwdSampleHist || MODE == kBorn) {
        const int cnt = (rx_range.x >= 0 && rx_range.y >= 0 && rx_range.x + rx_range.y <= p.n_rx) ? rx_range.y : 0;
        for (int e = tid; e < cnt; e += 128) {
            const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
            const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
            const int zn = node >> 16, xn = node & 0xffff;
            if (node < 0 || zn < z0 || zn >= z0 + TZ || xn < x0 || xn >= x0 + kTileX) {
                raise_status(p.status, DUFWI_ERR_GEOMETRY);
                continue;
            }
            p.cd[(static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r] =
                box[(zn - z0 + kVHalo) * kVBoxX + (xn - x0 + kVHalo)];
        }
    }
}

// ---- convolutional PML ------------------------------------------------------------------------
// The staggered operator of the variable-density step with each first difference stretched by
// one memory variable per axis (recursive convolution, coefficients a, b per node and half
// point from host tables):
//   psi^n = b psi^{n-1} + a D+u^n,  F = b_rho (D+u^n + psi^n),  xi^n = b xi^{n-1} + a D-F,
//   G = D-F + xi^n,  U^{n+1} = 2U^n - U^{n-1} + kappa' G  (no damping term; kappa' = rho C^2 dt^2/dx^2).
// The adjoint, written for mu = kappa' lambda, is the reverse of these statements: with chi and
// phi the adjoints of xi and psi,
//   e = mu^{n+1} + a (chi + mu^{n+1}),  chi <- b (chi + mu^{n+1}),  Fbar = -D+ e,
//   p = phi + b_rho Fbar,  dbar = b_rho Fbar + a p,  phi <- b p,
//   mu^n = 2 mu^{n+1} - mu^{n+2} - kappa' D- dbar (+ the scaled residual injections),
// and the imaging term is again mu^n G^{n-1} with G from the forward sweep's history.
// SO (0, or 1 + a second-order kind: kSoBorn with the forward arithmetic, kSoAdj and kSoBornAdj
// with the adjoint's) adds the second-order products' operands: Lap-history tiles t0, t1 in
// place of the history and sum tiles (the running sums are read from global memory).
template <int MODE, int SO = 0>
struct CpmlLayout {
    static constexpr bool kAdj = MODE == kAdjoint;
    static constexpr int kBox = kVBoxX * kVBoxZ;                  // 80 x 48
    static constexpr int kBx = kVFxX * kVTileZ;                   // 72 x 32 (x half points)
    static constexpr int kBz = kTileX * kVFzZ;                    // 64 x 40 (z half points)
    static constexpr int kTile = kTileX * kVTileZ;                // 64 x 32
    static constexpr int kNx = kAdj ? kVBoxX * kVTileZ : kTile;   // chi: 80 x 32; xi: 64 x 32
    static constexpr int kNz = kAdj ? kTileX * kVBoxZ : kTile;    // chi: 64 x 48; xi: 64 x 32
    static constexpr int kFloats = kBox + 2 * kBx + 2 * kBz + kNx + kNz + ((kAdj || SO) ? 4 : 2) * kTile;
    static constexpr uint32_t kBytes = kFloats * sizeof(float);
};

__device__ __forceinline__ float4 ldg4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// 128-bit global load with an evict-first L2 hint (data read once: the history).
__device__ __forceinline__ float4 ldg4_stream(const float *p)
{
#if DUFWI_L2_HINTS
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(l2_evict_first_policy()));
    return v;
#else
    return ldg4(p);
#endif
}

// (a, b) of a table of 4 rows of length n (a node, b node, a half, b half); identity outside.
__device__ __forceinline__ float2 cpml_coef(const float *t, int n, int row, int i)
{
    if (i < 0 || i >= n) return make_float2(0.f, 1.f);
    return make_float2(__ldg(t + (row + 0) * n + i), __ldg(t + (row + 1) * n + i));
}

// Second-order kinds (SO = 1 + kind; see so_step_kernel for the recursions), on the layer tiles:
//   kSoBorn (MODE kFwdHist): dU^{n+1} = the CPML step on dU (its own memory variables) + dkappa' G(U^n)
//     with G(U^n) from history slot q.h1_slot (tm.hist_tile) and dkappa' (tm.grad_tile, per map);
//     writes G(dU^n) to q.lap_out and samples dU^n into p.cd when given.
//   kSoAdj (MODE kAdjoint): the adjoint CPML step on mu; sums mu^m G(U^{m-1}) into q.sum1 and
//     mu^m G(dU^{m-1}) into q.sum2 (histories tm.hist_tile slot h1_slot, tm.grad_tile slot
//     h2_slot); writes its operator term A(mu^{m+1}) (mu^m = 2mu^{m+1} - mu^{m+2} + kappa' A) to
//     q.lap_out.
//   kSoBornAdj (MODE kAdjoint): the adjoint CPML step on dmu + dkappa' A(mu^{m+1}) (tm.grad_tile
//     per shot; dkappa' read from q.dkap); sums dmu^m G(U^{m-1}) into q.sum1.
template <int R, int MODE, int SO = 0>
__global__ void __launch_bounds__(128, 2)
cpml_step_kernel(const __grid_constant__ StepMaps tm, const __grid_constant__ CpmlMaps cm, const StepParams p,
                 const CpmlParams cp, const SoParams q)
{
    using CL = CpmlLayout<MODE, SO>;
    constexpr bool ADJ = CL::kAdj;
    constexpr int TZ = kVTileZ;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;
    __shared__ InjList inj;

    const int tid = threadIdx.x;
    const int s = p.shot0 + blockIdx.z;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * TZ;
    const int tx_idx = s % p.n_tx;
    const int map = s / p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *box = smem;                 // U^n (mu^{m+1}) with halo 8
    float *bxs = box + CL::kBox;       // buoyancy, x half points
    float *bzs = bxs + CL::kBx;        // buoyancy, z half points
    float *mhx = bzs + CL::kBz;        // psi / phi, x half points
    float *mhz = mhx + CL::kBx;        // psi / phi, z half points
    float *mnx = mhz + CL::kBz;        // xi / chi, x
    float *mnz = mnx + CL::kNx;        // xi / chi, z
    float *pv = mnz + CL::kNz;         // U^{n-1} (mu^{m+2})
    float *kp = pv + CL::kTile;        // kappa'
    float *hs = kp + CL::kTile;        // adjoint: G^{m-1} (second-order kinds: t0)
    float *gg = hs + CL::kTile;        // adjoint: imaging sums (second-order kinds: t1)
    if (x0 >= p.nxp || z0 >= p.nzp) return;
    if (p.tile_class == 2 && cpml_free_tile(p, x0, z0)) return;    // CPML split: interior tiles run elsewhere

    // early (as in the one-step kernel): buoyancies, U^{n-1}, kappa' and the history before the
    // wait; the memory variables come from the previous step and are requested after it
    if (tid == 0) {
        prefetch_tensormap(&tm.cur_box);
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, CL::kBytes);
        if (SO == 0 && p.early) {
            tma_load_3d(bxs, &tm.bx_tile, &bar, x0 - kHalo, z0, map);
            tma_load_3d(bzs, &tm.bz_tile, &bar, x0, z0 - kHalo, map);
            tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
            tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, map);
            if (ADJ) tma_load_4d_stream(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
        }
    }
    grid_dependency_wait();
    if (tid == 0) {
        tma_load_3d(box, &tm.cur_box, &bar, x0 - kVHalo, z0 - kVHalo, s);
        if (SO != 0 || !p.early) {
            tma_load_3d(bxs, &tm.bx_tile, &bar, x0 - kHalo, z0, map);
            tma_load_3d(bzs, &tm.bz_tile, &bar, x0, z0 - kHalo, map);
        }
        tma_load_3d(mhx, &cm.mem_hx, &bar, x0 - kHalo, z0, s);
        tma_load_3d(mhz, &cm.mem_hz, &bar, x0, z0 - kHalo, s);
        if (ADJ) {
            tma_load_3d(mnx, &cm.mem_nx, &bar, x0 - kVHalo, z0, s);
            tma_load_3d(mnz, &cm.mem_nz, &bar, x0, z0 - kVHalo, s);
        } else {
            tma_load_3d(mnx, &cm.mem_nx, &bar, x0, z0, s);
            tma_load_3d(mnz, &cm.mem_nz, &bar, x0, z0, s);
        }
        if (SO != 0) {
            tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
            tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, map);
            tma_load_4d(hs, &tm.hist_tile, &bar, x0, z0, s, q.h1_slot);
            if (SO == 1 + kSoBorn) tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, map);
            if (SO == 1 + kSoAdj) tma_load_4d(gg, &tm.grad_tile, &bar, x0, z0, s, q.h2_slot);
            if (SO == 1 + kSoBornAdj) tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, s);
        } else {
            if (!p.early) {
                tma_load_3d(pv, &tm.out_tile, &bar, x0, z0, s);
                tma_load_3d(kp, &tm.kap_tile, &bar, x0, z0, map);
                if (ADJ) tma_load_4d_stream(hs, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
            }
            if (ADJ) tma_load_3d(gg, &tm.grad_tile, &bar, x0, z0, s);
        }
    }
    grid_dependents_launch();

    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    int2 rx_range = make_int2(0, 0);
    if (MODE != kFwdHist || SO == 1 + kSoBorn) rx_range = __ldg(p.rx_tab + tx_idx * (gridDim.x * gridDim.y) + tile);
    if (SO == 1 + kSoBorn) {   // the Born field has no point source of its own
        if (tid == 0) inj.n = 0;
    } else {
        gather_injections<MODE>(inj, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX, TZ,
                                kTileX, tid, 128);
    }
    const int lx = (tid & 15) * 4;
    const int lz = (tid >> 4) * 4;
    const int gx = x0 + lx;
    const bool col_ok = gx < p.nxp;
    const int nxp = p.nxp, nzp = p.nzp;

    if (!wait_tile(&bar, p, tid)) return;

    float4 opv[4];     // forward: G; adjoint: -(D- dbar) along both axes
    float4 ctr[4];     // forward: U^n; adjoint: mu^{m+1} at the block
    // ---- x: rows lz .. lz + 3 of the block
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gz = z0 + lz + j;
        const bool row_ok = col_ok && gz < nzp;
        const long long orow = shot_off + static_cast<long long>(gz) * p.pitch + gx;
        float w[20];
        {
            const float *row = box + (lz + j + kVHalo) * kVBoxX + lx;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const float4 v = ld4s(row + 4 * c);
                w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
            }
        }
        ctr[j] = make_float4(w[8], w[9], w[10], w[11]);
        float bw[12], mw[12];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 b = ld4s(bxs + (lz + j) * kVFxX + lx + 4 * c);
            const float4 m = ld4s(mhx + (lz + j) * kVFxX + lx + 4 * c);
            bw[4 * c] = b.x; bw[4 * c + 1] = b.y; bw[4 * c + 2] = b.z; bw[4 * c + 3] = b.w;
            mw[4 * c] = m.x; mw[4 * c + 1] = m.y; mw[4 * c + 2] = m.z; mw[4 * c + 3] = m.w;
        }
        float ox[4];
        if (!ADJ) {
            float F[11], pn[4];
#pragma unroll
            for (int h = 0; h < 11; ++h) {
                float d = 0.0f;
#pragma unroll
                for (int k = 1; k <= R; ++k) d = fmaf(p.sw[k - 1], w[h + 4 + k] - w[h + 5 - k], d);
                const float2 ab = cpml_coef(cp.cx, nxp, 2, x0 - kHalo + lx + h);
                const float ps = fmaf(ab.y, mw[h], ab.x * d);
                F[h] = bw[h] * (d + ps);
                if (h >= 4 && h < 8) pn[h - 4] = ps;
            }
            const float4 xi_prev = ld4s(mnx + (lz + j) * kTileX + lx);
            const float xp[4] = {xi_prev.x, xi_prev.y, xi_prev.z, xi_prev.w};
            float xn[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float e = 0.0f;
#pragma unroll
                for (int k = 1; k <= R; ++k) e = fmaf(p.sw[k - 1], F[q + k + 3] - F[q - k + 4], e);
                const float2 ab = cpml_coef(cp.cx, nxp, 0, gx + q);
                xn[q] = fmaf(ab.y, xp[q], ab.x * e);
                ox[q] = e + xn[q];
            }
            if (row_ok) {
                float4 a = make_float4(pn[0], pn[1], pn[2], pn[3]), b = make_float4(xn[0], xn[1], xn[2], xn[3]);
                if (gx + 4 > nxp) {
                    if (gx + 1 >= nxp) { a.y = 0.f; b.y = 0.f; }
                    if (gx + 2 >= nxp) { a.z = 0.f; b.z = 0.f; }
                    a.w = 0.f; b.w = 0.f;
                }
                st4(cp.hx_out + orow, a);
                st4(cp.nx_out + orow, b);
            }
        } else {
            float cw[20];
            {
                const float *row = mnx + (lz + j) * kVBoxX + lx;
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const float4 v = ld4s(row + 4 * c);
                    cw[4 * c] = v.x; cw[4 * c + 1] = v.y; cw[4 * c + 2] = v.z; cw[4 * c + 3] = v.w;
                }
            }
            float e[20];
#pragma unroll
            for (int c = 0; c < 20; ++c) {
                const float2 ab = cpml_coef(cp.cx, nxp, 0, x0 - kVHalo + lx + c);
                e[c] = fmaf(ab.x, cw[c] + w[c], w[c]);
            }
            float db[11], pn[4];
#pragma unroll
            for (int h = 0; h < 11; ++h) {
                float fb = 0.0f;
#pragma unroll
                for (int k = 1; k <= R; ++k) fb = fmaf(p.sw[k - 1], e[h + 5 - k] - e[h + 4 + k], fb);
                const float2 ab = cpml_coef(cp.cx, nxp, 2, x0 - kHalo + lx + h);
                const float bf = bw[h] * fb;
                const float pp = mw[h] + bf;
                db[h] = fmaf(ab.x, pp, bf);
                if (h >= 4 && h < 8) pn[h - 4] = ab.y * pp;
            }
            float cn[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 1; k <= R; ++k) acc = fmaf(p.sw[k - 1], db[q + 4 - k] - db[q + 3 + k], acc);
                ox[q] = acc;
                const float2 ab = cpml_coef(cp.cx, nxp, 0, gx + q);
                cn[q] = ab.y * (cw[8 + q] + w[8 + q]);
            }
            if (row_ok) {
                float4 a = make_float4(pn[0], pn[1], pn[2], pn[3]), b = make_float4(cn[0], cn[1], cn[2], cn[3]);
                if (gx + 4 > nxp) {
                    if (gx + 1 >= nxp) { a.y = 0.f; b.y = 0.f; }
                    if (gx + 2 >= nxp) { a.z = 0.f; b.z = 0.f; }
                    a.w = 0.f; b.w = 0.f;
                }
                st4(cp.hx_out + orow, a);
                st4(cp.nx_out + orow, b);
            }
        }
        opv[j] = make_float4(ox[0], ox[1], ox[2], ox[3]);
    }
    // ---- z: columns lx .. lx + 3 of the block
    {
        float4 col[18];
#pragma unroll
        for (int r = 0; r < 18; ++r) col[r] = ld4s(box + (lz + 1 + r) * kVBoxX + lx + kVHalo);
        float4 oz[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) oz[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!ADJ) {
#pragma unroll
            for (int f = 0; f < 11; ++f) {
                float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                    const float4 up = col[f + 3 + k], dn = col[f + 4 - k];
                    const float sk = p.sw[k - 1];
                    d.x = fmaf(sk, up.x - dn.x, d.x);
                    d.y = fmaf(sk, up.y - dn.y, d.y);
                    d.z = fmaf(sk, up.z - dn.z, d.z);
                    d.w = fmaf(sk, up.w - dn.w, d.w);
                }
                const float2 ab = cpml_coef(cp.cz, nzp, 2, z0 - kHalo + lz + f);
                const float4 m = ld4s(mhz + (lz + f) * kTileX + lx);
                const float4 ps = make_float4(fmaf(ab.y, m.x, ab.x * d.x), fmaf(ab.y, m.y, ab.x * d.y),
                                              fmaf(ab.y, m.z, ab.x * d.z), fmaf(ab.y, m.w, ab.x * d.w));
                const float4 b = ld4s(bzs + (lz + f) * kTileX + lx);
                const float4 fl = make_float4(b.x * (d.x + ps.x), b.y * (d.y + ps.y), b.z * (d.z + ps.z),
                                              b.w * (d.w + ps.w));
                if (f >= 4 && f < 8) {
                    const int gz = z0 + lz + f - 4;
                    if (col_ok && gz < nzp) {
                        float4 v = ps;
                        if (gx + 4 > nxp) {
                            if (gx + 1 >= nxp) v.y = 0.f;
                            if (gx + 2 >= nxp) v.z = 0.f;
                            v.w = 0.f;
                        }
                        st4(cp.hz_out + shot_off + static_cast<long long>(gz) * p.pitch + gx, v);
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int kp_ = f - j - 3, km_ = j + 4 - f;
                    if (kp_ >= 1 && kp_ <= R) oz[j] = fma4(make_float4(p.sw[kp_ - 1], p.sw[kp_ - 1], p.sw[kp_ - 1],
                                                                       p.sw[kp_ - 1]), fl, oz[j]);
                    if (km_ >= 1 && km_ <= R) oz[j] = fma4(make_float4(-p.sw[km_ - 1], -p.sw[km_ - 1],
                                                                       -p.sw[km_ - 1], -p.sw[km_ - 1]), fl, oz[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gz = z0 + lz + j;
                const float2 ab = cpml_coef(cp.cz, nzp, 0, gz);
                const float4 xp = ld4s(mnz + (lz + j) * kTileX + lx);
                float4 xn = make_float4(fmaf(ab.y, xp.x, ab.x * oz[j].x), fmaf(ab.y, xp.y, ab.x * oz[j].y),
                                        fmaf(ab.y, xp.z, ab.x * oz[j].z), fmaf(ab.y, xp.w, ab.x * oz[j].w));
                opv[j] = make_float4(opv[j].x + (oz[j].x + xn.x), opv[j].y + (oz[j].y + xn.y),
                                     opv[j].z + (oz[j].z + xn.z), opv[j].w + (oz[j].w + xn.w));
                if (col_ok && gz < nzp) {
                    if (gx + 4 > nxp) {
                        if (gx + 1 >= nxp) xn.y = 0.f;
                        if (gx + 2 >= nxp) xn.z = 0.f;
                        xn.w = 0.f;
                    }
                    st4(cp.nz_out + shot_off + static_cast<long long>(gz) * p.pitch + gx, xn);
                }
            }
        } else {
            // e at node rows lz + 1 .. lz + 18 of the box, chi from its 64 x 48 box (same rows)
            float4 e[18];
#pragma unroll
            for (int r = 0; r < 18; ++r) {
                const float4 c = ld4s(mnz + (lz + 1 + r) * kTileX + lx);
                const float a = cpml_coef(cp.cz, nzp, 0, z0 - kVHalo + lz + 1 + r).x;
                e[r] = make_float4(fmaf(a, c.x + col[r].x, col[r].x), fmaf(a, c.y + col[r].y, col[r].y),
                                   fmaf(a, c.z + col[r].z, col[r].z), fmaf(a, c.w + col[r].w, col[r].w));
            }
#pragma unroll
            for (int f = 0; f < 11; ++f) {
                float4 fb = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                    const float4 a = e[f + 4 - k], b = e[f + 3 + k];
                    const float sk = p.sw[k - 1];
                    fb.x = fmaf(sk, a.x - b.x, fb.x);
                    fb.y = fmaf(sk, a.y - b.y, fb.y);
                    fb.z = fmaf(sk, a.z - b.z, fb.z);
                    fb.w = fmaf(sk, a.w - b.w, fb.w);
                }
                const float2 ab = cpml_coef(cp.cz, nzp, 2, z0 - kHalo + lz + f);
                const float4 b = ld4s(bzs + (lz + f) * kTileX + lx);
                const float4 m = ld4s(mhz + (lz + f) * kTileX + lx);
                const float4 bf = make_float4(b.x * fb.x, b.y * fb.y, b.z * fb.z, b.w * fb.w);
                const float4 pp = make_float4(m.x + bf.x, m.y + bf.y, m.z + bf.z, m.w + bf.w);
                const float4 db = make_float4(fmaf(ab.x, pp.x, bf.x), fmaf(ab.x, pp.y, bf.y), fmaf(ab.x, pp.z, bf.z),
                                              fmaf(ab.x, pp.w, bf.w));
                if (f >= 4 && f < 8) {
                    const int gz = z0 + lz + f - 4;
                    if (col_ok && gz < nzp) {
                        float4 v = make_float4(ab.y * pp.x, ab.y * pp.y, ab.y * pp.z, ab.y * pp.w);
                        if (gx + 4 > nxp) {
                            if (gx + 1 >= nxp) v.y = 0.f;
                            if (gx + 2 >= nxp) v.z = 0.f;
                            v.w = 0.f;
                        }
                        st4(cp.hz_out + shot_off + static_cast<long long>(gz) * p.pitch + gx, v);
                    }
                }
                // out_j = sum_k s_k (dbar_{j+4-k} - dbar_{j+3+k})
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int kp_ = j + 4 - f, km_ = f - j - 3;
                    if (kp_ >= 1 && kp_ <= R) oz[j] = fma4(make_float4(p.sw[kp_ - 1], p.sw[kp_ - 1], p.sw[kp_ - 1],
                                                                       p.sw[kp_ - 1]), db, oz[j]);
                    if (km_ >= 1 && km_ <= R) oz[j] = fma4(make_float4(-p.sw[km_ - 1], -p.sw[km_ - 1],
                                                                       -p.sw[km_ - 1], -p.sw[km_ - 1]), db, oz[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gz = z0 + lz + j;
                const float b = cpml_coef(cp.cz, nzp, 0, gz).y;
                const float4 c = ld4s(mnz + (lz + 8 + j) * kTileX + lx);
                const float4 m = col[7 + j];
                float4 cn = make_float4(b * (c.x + m.x), b * (c.y + m.y), b * (c.z + m.z), b * (c.w + m.w));
                opv[j] = make_float4(opv[j].x + oz[j].x, opv[j].y + oz[j].y, opv[j].z + oz[j].z, opv[j].w + oz[j].w);
                if (col_ok && gz < nzp) {
                    if (gx + 4 > nxp) {
                        if (gx + 1 >= nxp) cn.y = 0.f;
                        if (gx + 2 >= nxp) cn.z = 0.f;
                        cn.w = 0.f;
                    }
                    st4(cp.nz_out + shot_off + static_cast<long long>(gz) * p.pitch + gx, cn);
                }
            }
        }
    }
    // ---- update: U^{n+1} = 2U^n - U^{n-1} + kappa' G  (adjoint: mu^m = 2mu^{m+1} - mu^{m+2} + kappa' out)
    float4 nxt[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int lo = (lz + j) * kTileX + lx;
        const float4 pp = ld4s(pv + lo), kk = ld4s(kp + lo), u = ctr[j];
        nxt[j] = fma4(kk, opv[j], make_float4(2.f * u.x - pp.x, 2.f * u.y - pp.y, 2.f * u.z - pp.z, 2.f * u.w - pp.w));
        if (SO == 1 + kSoBorn) nxt[j] = fma4(ld4s(gg + lo), ld4s(hs + lo), nxt[j]);          // + dkappa' G(U^n)
        if (SO == 1 + kSoBornAdj) {                                                          // + dkappa' A(mu^{m+1})
            const int gz = z0 + lz + j;
            const float4 dk = (col_ok && gz < nzp)
                                  ? ldg4(q.dkap + static_cast<long long>(map) * p.slice +
                                         static_cast<long long>(gz) * p.pitch + gx)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            nxt[j] = fma4(dk, ld4s(gg + lo), nxt[j]);
        }
    }
    if (inj.n > 0) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) st4s(pv + (lz + j) * kTileX + lx, nxt[j]);
        __syncthreads();
        if (tid == 0)
            apply_injections<MODE>(inj, pv, p, p.rx_sorted, p.n_rx, s, tx_idx, p.step, rx_range, x0, z0, kTileX, TZ,
                                   kTileX);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) nxt[j] = ld4s(pv + (lz + j) * kTileX + lx);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gz = z0 + lz + j;
        if (!col_ok || gz >= nzp) continue;
        float4 nv = nxt[j], lv = opv[j];
        if (gx + 4 > nxp) {
            if (gx + 1 >= nxp) { nv.y = 0.f; lv.y = 0.f; }
            if (gx + 2 >= nxp) { nv.z = 0.f; lv.z = 0.f; }
            nv.w = 0.f; lv.w = 0.f;
        }
        const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
        const int lo = (lz + j) * kTileX + lx;
        st4(p.out + o, nv);
        if (SO == 0) {
            if (MODE == kFwdSampleHist || MODE == kFwdHist) st4_stream(p.hist + o, lv);
            if (MODE == kAdjoint) st4(p.grad + o, fma4(nv, ld4s(hs + lo), ld4s(gg + lo)));
        } else {
            if (SO == 1 + kSoBorn || SO == 1 + kSoAdj) st4(q.lap_out + o, lv);
            if (SO == 1 + kSoAdj) {
                st4(q.sum1 + o, fma4(nv, ld4s(hs + lo), ldg4(q.sum1 + o)));
                st4(q.sum2 + o, fma4(nv, ld4s(gg + lo), ldg4(q.sum2 + o)));
            }
            if (SO == 1 + kSoBornAdj) st4(q.sum1 + o, fma4(nv, ld4s(hs + lo), ldg4(q.sum1 + o)));
        }
    }
    if (MODE == kFwdSample || MODE == kFwdSampleHist || (SO == 1 + kSoBorn && p.cd)) {
        const int cnt = (rx_range.x >= 0 && rx_range.y >= 0 && rx_range.x + rx_range.y <= p.n_rx) ? rx_range.y : 0;
        for (int e = tid; e < cnt; e += 128) {
            const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
            const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
            const int zn = node >> 16, xn = node & 0xffff;
            if (node < 0 || zn < z0 || zn >= z0 + TZ || xn < x0 || xn >= x0 + kTileX) {
                raise_status(p.status, DUFWI_ERR_GEOMETRY);
                continue;
            }
            p.cd[(static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r] =
                box[(zn - z0 + kVHalo) * kVBoxX + (xn - x0 + kVHalo)];
        }
    }
}

// ---- cluster-resident sweep --------------------------------------------------------------------
// For small grids (one shot's fields in the shared memory of kClusterCtas CTAs) a whole range of
// steps runs in one launch of one cluster per shot. CTA rank k holds rows [k H, (k + 1) H) of the
// padded grid in three rotating field buffers (the field being read, with 4 halo rows on each
// side; the previous one; the one being written), kappa' and, in the adjoint, the imaging sum.
// Each step: copy the halo rows of the field being read from the neighbours' buffers through
// distributed shared memory, update the owned rows with the one-step kernel's arithmetic (the same
// Laplacian and Eq. 2 operations in the same order, so the results are bit-identical), apply the
// point injections in list order, write the history and traces, and synchronise the cluster. The
// buffer written at step i is read by the neighbours at step i + 1 and overwritten only at step
// i + 3, after two more cluster barriers, so one barrier per step suffices. Every CTA runs every
// barrier (no early exit), so the cluster cannot stall on a missing arrival.

// lap_block with a run-time row stride (identical operations).
template <int R>
__device__ __forceinline__ void lap_block_rs(const float *src, int sx, int cx, int cz, const float *c,
                                             float4 (&lap)[4], float4 (&ctr)[4])
{
    float4 col[4 + 2 * R];
#pragma unroll
    for (int i = 0; i < 4 + 2 * R; ++i) col[i] = ld4s(src + (cz - R + i) * sx + cx);
    const float2 m4 = make_float2(-4.0f, -4.0f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 lft = ld4s(src + (cz + j) * sx + cx - 4);
        const float4 rgt = ld4s(src + (cz + j) * sx + cx + 4);
        const float4 cc = col[R + j];
        ctr[j] = cc;
        const float w[12] = {lft.x, lft.y, lft.z, lft.w, cc.x, cc.y, cc.z, cc.w, rgt.x, rgt.y, rgt.z, rgt.w};
        float2 l[2];
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
                acc = __ffma2_rn(make_float2(c[kk], c[kk]), __fadd2_rn(__fadd2_rn(xs, zs), nu4), acc);
            }
            l[h] = acc;
        }
        lap[j] = make_float4(l[0].x, l[0].y, l[1].x, l[1].y);
    }
}

constexpr int kClusterThreads = 256;

constexpr int kClusterList = 128;   // receivers (or the source) inside one CTA's strip

template <int R, int MODE>
__global__ void __launch_bounds__(kClusterThreads, 1)
cluster_sweep_kernel(const StepParams p, const ClusterParams cp)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(128) float smem[];
    // receivers sampled (forward) and point injections (source or receivers) inside this strip:
    // buffer index and receiver number, in list order; the injection values of the current step
    __shared__ int smp_idx[kClusterList], smp_r[kClusterList], inj_idx[kClusterList], inj_r[kClusterList];
    __shared__ float inj_v[kClusterList];
    __shared__ int n_smp, n_inj;
    const int tid = threadIdx.x;
    const int rank = static_cast<int>(cl.block_rank());
    const int s = p.shot0 + blockIdx.y;
    const int tx_idx = s % p.n_tx;
    const int map = s / p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    const int H = cp.H, lp = cp.lpitch, nxp = p.nxp, nzp = p.nzp;
    const int z_lo = rank * H;                                  // first owned row
    const int rows = max(0, min(H, nzp - z_lo));                // owned rows inside the grid
    const int fsz = (H + 8) * lp;                               // one field buffer, halo rows included
    float *F[3] = {smem, smem + fsz, smem + 2 * fsz};
    float *kap = smem + 3 * fsz;                                // H x lp
    float *G = kap + H * lp;                                    // adjoint imaging sum, H x lp
    const int nq = (nxp + 3) / 4;                               // float4 columns of a row
    const MapGrid mg = map_grid(p, map);
    auto in_strip = [&](int node, int &idx) {
        const int zn = node >> 16, xn = node & 0xffff;
        if (node < 0 || zn >= nzp || xn >= nxp) {
            if (rank == 0) raise_status(p.status, DUFWI_ERR_GEOMETRY);
            return false;
        }
        idx = (zn - z_lo + 4) * lp + 4 + xn;
        return zn >= z_lo && zn < z_lo + rows;
    };

    // zero everything (halo rows outside the grid and pad columns stay zero), then load the owned
    // rows of U^{n0} (buffer 0), U^{n0-1} (buffer 2), kappa' and the running imaging sum
    for (int i = tid; i < (3 * fsz + 2 * H * lp) / 4; i += kClusterThreads)
        reinterpret_cast<float4 *>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0) {   // the strip's receivers and injections, in list order
        int m = 0, k = 0, idx = 0;
        if ((MODE == kFwdSample || MODE == kFwdSampleHist) && p.cd)
            for (int r = 0; r < p.n_rx; ++r)
                if (in_strip(__ldg(p.smp_node + tx_idx * p.n_rx + r), idx)) {
                    if (m < kClusterList) { smp_idx[m] = idx; smp_r[m] = r; }
                    ++m;
                }
        if (MODE == kAdjoint) {
            for (int r = 0; r < p.n_rx; ++r)
                if (in_strip(__ldg(p.inj_node + tx_idx * p.n_rx + r), idx)) {
                    if (k < kClusterList) { inj_idx[k] = idx; inj_r[k] = r; }
                    ++k;
                }
        } else if (in_strip(__ldg(p.inj_node + tx_idx), idx)) {
            inj_idx[0] = idx;
            inj_r[0] = 0;
            k = 1;
        }
        if (m > kClusterList || k > kClusterList) raise_status(p.status, DUFWI_ERR_UNSUPPORTED);
        n_smp = min(m, kClusterList);
        n_inj = min(k, kClusterList);
    }
    __syncthreads();
    for (int i = tid; i < rows * nq; i += kClusterThreads) {
        const int r = i / nq, q4 = (i - r * nq) * 4;
        const long long g = shot_off + static_cast<long long>(z_lo + r) * p.pitch + q4;
        st4s(F[0] + (r + 4) * lp + 4 + q4, ldg4(cp.cur + g));
        st4s(F[2] + (r + 4) * lp + 4 + q4, ldg4(cp.prv + g));
        st4s(kap + r * lp + 4 + q4,
             ldg4(p.kap + static_cast<long long>(map) * p.slice + static_cast<long long>(z_lo + r) * p.pitch + q4));
        if (MODE == kAdjoint) st4s(G + r * lp + 4 + q4, ldg4(p.grad + g));
    }
    cl.sync();

    constexpr int kHReg = 8;                                    // history prefetch: float4 per thread
    const bool hreg_ok = rows * nq <= kHReg * kClusterThreads;
    int ci = 0;                                                 // F[ci] holds the field being read
    for (int i = 0; i < cp.n_steps; ++i) {
        const int step = MODE == kAdjoint ? cp.step0 - i : cp.step0 + i;
        float *cur = F[ci], *prv = F[(ci + 2) % 3], *out = F[(ci + 1) % 3];
        // requests that do not depend on this step's arithmetic go first: the history rows the
        // imaging reads (adjoint), this step's injection values, the traces of U^n
        float4 hreg[kHReg];
        const float *hm = cp.hist0 - static_cast<long long>(i) * cp.hist_stride + shot_off;
        if (MODE == kAdjoint && hreg_ok) {
#pragma unroll
            for (int j = 0; j < kHReg; ++j) {
                const int e = tid + j * kClusterThreads;
                if (e < rows * nq) {
                    const int r = e / nq, q4 = (e - r * nq) * 4;
                    hreg[j] = ldg4_stream(hm + static_cast<long long>(z_lo + r) * p.pitch + q4);
                }
            }
        }
        if (tid < n_inj) {
            inj_v[tid] = MODE == kAdjoint
                ? __ldg(p.inj_val + (static_cast<long long>(s) * p.nt + step) * p.n_rx + inj_r[tid])
                : __fmul_rn(p.inj_scale, __ldg(p.inj_val + static_cast<long long>(p.wav_per_tx ? tx_idx : 0) * p.nt + step));
        }
        if (tid < n_smp) p.cd[(static_cast<long long>(s) * p.nt + step) * p.n_rx + smp_r[tid]] = cur[smp_idx[tid]];
        // halo rows of cur from the neighbours (rows outside the grid stay zero)
        if (rank > 0) {
            const float *up = cl.map_shared_rank(cur, rank - 1);
            for (int e = tid; e < 4 * (lp / 4); e += kClusterThreads) {
                const int r = e / (lp / 4), q4 = (e - r * (lp / 4)) * 4;
                st4s(cur + r * lp + q4, *reinterpret_cast<const float4 *>(up + (H + r) * lp + q4));
            }
        }
        if (rank + 1 < static_cast<int>(cl.num_blocks()) && z_lo + H < nzp) {
            const float *dn = cl.map_shared_rank(cur, rank + 1);
            for (int e = tid; e < 4 * (lp / 4); e += kClusterThreads) {
                const int r = e / (lp / 4), q4 = (e - r * (lp / 4)) * 4;
                st4s(cur + (H + 4 + r) * lp + q4, *reinterpret_cast<const float4 *>(dn + (4 + r) * lp + q4));
            }
        }
        __syncthreads();
        // update of the owned rows (blocks of 4 x 4; at the grid's last rows the block rows past
        // nzp are computed and not stored)
        const int nbr = (rows + 3) / 4;
        for (int b = tid; b < nbr * nq; b += kClusterThreads) {
            const int br = b / nq, bq = b - br * nq;
            const int lz = 4 + 4 * br, lx = 4 + 4 * bq;
            const int gz0 = z_lo + 4 * br, gx = 4 * bq;
            float4 lap[4], ctr[4];
            lap_block_rs<R>(cur, lp, lx, lz, p.c, lap, ctr);
            const bool interior = region_interior(p, mg, gx, gz0, 4, 4);
            int xd[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) xd[k] = layer_depth(gx + k, p.P, mg.Nx);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gz = gz0 + j;
                if (gz >= z_lo + rows) continue;
                const int lo = (lz + j) * lp + lx;
                float4 nv = eq2_row(ctr[j], ld4s(prv + lo), ld4s(kap + (lz + j - 4) * lp + lx), lap[j], interior,
                                    p.damp_tab + layer_depth(gz, p.P, mg.Nz) * (p.P + 1), xd);
                float4 lv = lap[j];
                if (gx + 4 > nxp) {   // lanes past the last column stay zero (outside the grid)
                    if (gx + 1 >= nxp) { nv.y = 0.f; lv.y = 0.f; }
                    if (gx + 2 >= nxp) { nv.z = 0.f; lv.z = 0.f; }
                    nv.w = 0.f; lv.w = 0.f;
                }
                st4s(out + lo, nv);
                if (MODE == kFwdSampleHist || MODE == kFwdHist)
                    st4_stream(cp.hist0 + static_cast<long long>(i) * cp.hist_stride + shot_off +
                               static_cast<long long>(gz) * p.pitch + gx, lv);
            }
        }
        __syncthreads();
        // point injections of this step, in list order (thread 0): the product was rounded
        // before the add, as in the one-step kernel
        if (tid == 0)
            for (int e = 0; e < n_inj; ++e) out[inj_idx[e]] = __fadd_rn(out[inj_idx[e]], inj_v[e]);
        if (MODE == kAdjoint) {   // imaging: G += mu^m Lap(U^{m-1}), with mu^m after the injections
            __syncthreads();
            if (hreg_ok) {
#pragma unroll
                for (int j = 0; j < kHReg; ++j) {
                    const int e = tid + j * kClusterThreads;
                    if (e < rows * nq) {
                        const int r = e / nq, q4 = (e - r * nq) * 4;
                        float *gp = G + r * lp + 4 + q4;
                        st4s(gp, fma4(ld4s(out + (r + 4) * lp + 4 + q4), hreg[j], ld4s(gp)));
                    }
                }
            } else {
                for (int e = tid; e < rows * nq; e += kClusterThreads) {
                    const int r = e / nq, q4 = (e - r * nq) * 4;
                    float *gp = G + r * lp + 4 + q4;
                    st4s(gp, fma4(ld4s(out + (r + 4) * lp + 4 + q4),
                                  ldg4(hm + static_cast<long long>(z_lo + r) * p.pitch + q4), ld4s(gp)));
                }
            }
        }
        cl.sync();
        ci = (ci + 1) % 3;
    }
    // the last two fields (and the imaging sum) back to global memory
    const float *fc = F[ci], *fp = F[(ci + 2) % 3];
    for (int i = tid; i < rows * nq; i += kClusterThreads) {
        const int r = i / nq, q4 = (i - r * nq) * 4;
        const long long g = shot_off + static_cast<long long>(z_lo + r) * p.pitch + q4;
        st4(cp.out_cur + g, ld4s(fc + (r + 4) * lp + 4 + q4));
        st4(cp.out_prv + g, ld4s(fp + (r + 4) * lp + 4 + q4));
        if (MODE == kAdjoint) st4(p.grad + g, ld4s(G + r * lp + 4 + q4));
    }
    // no CTA leaves while a neighbour may still read its buffers
    cl.sync();
}

// ---- persistent sweep ---------------------------------------------------------------------------
// Several time steps of one sweep in one cooperative launch (see SweepParams). Each work item is
// the one-step update of one 64 x 32 tile; the arithmetic is that of step_kernel<R, MODE, 32>, so
// the results are bit-identical. Ordering between CTAs: the producer's threads store the tile,
// the CTA barrier orders those stores before thread 0's release of the tile counter; a consumer's
// thread 0 acquires the counters of the tile and its four neighbours, then a proxy fence orders
// that acquire before its TMA (async proxy) reads. Counter waits are bounded like the mbarrier
// waits: a CTA whose wait runs out raises DUFWI_ERR_TIMEOUT, sets the abort word and returns, and
// every other waiter returns when it sees the abort word.
__device__ __forceinline__ void st_release(int *ptr, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(ptr), "r"(v) : "memory");
}


__device__ __forceinline__ int ld_relaxed(const int *ptr)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(ptr) : "memory");
    return v;
}

// Thread 0: waits until the counters of tile k and its in-shot neighbours reach target; false on
// abort or timeout (the abort word is then set). The up to five counters are read together with
// relaxed loads (one round trip to L2 per poll); the fence after the last poll makes the reads
// an acquire pattern with the producers' releases.
__device__ bool wait_neighbours(const SweepParams &sp, int k, int target, int *status)
{
    if (k == sp.stall_tile) target = 0x7fffffff;   // test hook: a counter value nothing reaches
    const int per_shot = sp.tiles_x * sp.tiles_z;
    const int t = k % per_shot, tx = t % sp.tiles_x, tz = t / sp.tiles_x;
    const int kl = tx > 0 ? k - 1 : k;
    const int kr = tx + 1 < sp.tiles_x ? k + 1 : k;
    const int ku = tz > 0 ? k - sp.tiles_x : k;
    const int kd = tz + 1 < sp.tiles_z ? k + sp.tiles_x : k;
    unsigned long long t0 = 0;
    for (unsigned polls = 0;; ++polls) {
        const int a = ld_relaxed(sp.flags + k), b = ld_relaxed(sp.flags + kl), c = ld_relaxed(sp.flags + kr);
        const int e = ld_relaxed(sp.flags + ku), f = ld_relaxed(sp.flags + kd);
        if (min(min(a, b), min(min(c, e), f)) >= target) break;
        if ((polls & 31) == 31) {   // abort word and time limit every 32 polls
            if (ld_relaxed(sp.abort) != 0) return false;
            const unsigned long long now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitLimitNs) {
                raise_status(status, DUFWI_ERR_TIMEOUT);
                st_release(sp.abort, 1);
                return false;
            }
        }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
}

template <int R, int MODE>
__global__ void __launch_bounds__(128, DUFWI_STEP_MIN_CTAS_128)
sweep_kernel(const __grid_constant__ SweepMaps tm, const StepParams p, const SweepParams sp)
{
    using TL = TileLayout<MODE, 32>;
    constexpr int TZ = 32;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;
    __shared__ InjList inj;
    __shared__ int go;

    const int tid = threadIdx.x;
    float *box = smem;
    float *pv = box + TL::kBox;
    float *kp = pv + TL::kTile;
    float *hs = kp + TL::kTile;
    float *gg = hs + TL::kTile;
    const int per_shot = sp.tiles_x * sp.tiles_z;
    const int n_items = sp.n_steps * sp.tiles;   // < 2^31 (checked on the host)
    if (tid == 0) {
        prefetch_tensormap(&tm.box[0]);
        prefetch_tensormap(&tm.box[1]);
        mbar_init(&bar, 1);
    }
    __syncthreads();
    const int lx = (tid & 15) * 4;
    const int lz = (tid >> 4) * 4;
    uint32_t parity = 0;
#pragma unroll 1
    for (int g = blockIdx.x; g < n_items; g += gridDim.x) {
        const int i = g / sp.tiles;
        const int k = g - i * sp.tiles;
        const int s = k / per_shot;
        const int t = k % per_shot;
        const int x0 = (t % sp.tiles_x) * kTileX;
        const int z0 = (t / sp.tiles_x) * TZ;
        const int tx_idx = s % p.n_tx;
        const int map = s / p.n_tx;
        const int step = MODE == kAdjoint ? sp.step0 - i : sp.step0 + i;
        const MapGrid mg = map_grid(p, map);
        const bool active = x0 < mg.nxp && z0 < mg.nzp;   // sized calls: tiles outside the map stay zero
        float *out = (i & 1) ? sp.out[1] : sp.out[0];

        if (tid == 0) {
            const int ok = wait_neighbours(sp, k, i, p.status) ? 1 : 0;
            if (ok && active) {
                fence_proxy_async_global();    // acquired stores of other CTAs, before the TMA reads
                fence_proxy_async_shared();    // this CTA's earlier shared-memory use, before the TMA writes
                mbar_arrive_expect_tx(&bar, TL::kBytes);
                tma_load_3d(box, &tm.box[i & 1], &bar, x0 - kHalo, z0 - kHalo, s);
                tma_load_3d(pv, &tm.tile[i & 1], &bar, x0, z0, s);
                tma_load_3d(kp, &tm.kap, &bar, x0, z0, map);
                if (MODE == kAdjoint) {
                    tma_load_4d(hs, &tm.hist, &bar, x0, z0, s, sp.hist_slot0 - i);
                    tma_load_3d(gg, &tm.grad, &bar, x0, z0, s);
                }
            }
            go = ok;
        }
        __syncthreads();
        if (!go) return;
        if (active) {
            int2 rx_range = make_int2(0, 0);
            if (MODE != kFwdHist) rx_range = __ldg(p.rx_tab + tx_idx * per_shot + t);
            gather_injections<MODE>(inj, p, p.rx_sorted, p.n_rx, s, tx_idx, step, rx_range, x0, z0, kTileX, TZ,
                                    kTileX, tid, 128);
            const int gx = x0 + lx;
            const bool interior = region_interior(p, mg, x0, z0, kTileX, TZ);
            int xd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) xd[q] = layer_depth(gx + q, p.P, mg.Nx);

            // bounded wait on this item's phase (thread 0 polls, the CTA barrier publishes the result)
            int fail = 0;
            if (tid == 0) fail = !mbar_wait_bounded(&bar, parity);
            if (__syncthreads_or(fail)) {
                if (tid == 0) {
                    raise_status(p.status, DUFWI_ERR_TIMEOUT);
                    st_release(sp.abort, 1);
                    mbar_wait_bounded(&bar, parity);
                }
                return;
            }
            if (!mbar_try_wait_sleep(&bar, parity) && !mbar_wait_bounded(&bar, parity))
                raise_status(p.status, DUFWI_ERR_TIMEOUT);
            parity ^= 1u;

            float4 lap[4], ctr[4], nxt[4];
            lap_block<R, kBoxX>(box, kHalo + lx, kHalo + lz, p.c, lap, ctr);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int lo = (lz + j) * kTileX + lx;
                nxt[j] = eq2_row(ctr[j], ld4s(pv + lo), ld4s(kp + lo), lap[j], interior,
                                 p.damp_tab + layer_depth(z0 + lz + j, p.P, mg.Nz) * (p.P + 1), xd);
            }
            if (inj.n > 0) {
                __syncthreads();
#pragma unroll
                for (int j = 0; j < 4; ++j) st4s(pv + (lz + j) * kTileX + lx, nxt[j]);
                __syncthreads();
                if (tid == 0)
                    apply_injections<MODE>(inj, pv, p, p.rx_sorted, p.n_rx, s, tx_idx, step, rx_range, x0, z0, kTileX,
                                           TZ, kTileX);
                __syncthreads();
#pragma unroll
                for (int j = 0; j < 4; ++j) nxt[j] = ld4s(pv + (lz + j) * kTileX + lx);
            }
            const bool col_ok = gx < mg.nxp;
            const long long shot_off = static_cast<long long>(s) * p.slice;
            float *hist = (MODE == kFwdSampleHist || MODE == kFwdHist) ? sp.hist0 + sp.hist_stride * i : nullptr;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gz = z0 + lz + j;
                if (!col_ok || gz >= mg.nzp) continue;
                float4 nv = nxt[j], lv = lap[j];
                if (gx + 4 > mg.nxp) {
                    if (gx + 1 >= mg.nxp) { nv.y = 0.f; lv.y = 0.f; }
                    if (gx + 2 >= mg.nxp) { nv.z = 0.f; lv.z = 0.f; }
                    nv.w = 0.f; lv.w = 0.f;
                }
                const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
                st4(out + o, nv);
                if (MODE == kFwdSampleHist || MODE == kFwdHist) st4(hist + o, lv);
                if (MODE == kAdjoint) {
                    const int lo = (lz + j) * kTileX + lx;
                    st4(p.grad + o, fma4(nv, ld4s(hs + lo), ld4s(gg + lo)));
                }
            }
            if (MODE == kFwdSample || MODE == kFwdSampleHist) {
                const int cnt =
                    (rx_range.x >= 0 && rx_range.y >= 0 && rx_range.x + rx_range.y <= p.n_rx) ? rx_range.y : 0;
                for (int e = tid; e < cnt; e += 128) {
                    const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
                    const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
                    const int zn = node >> 16, xn = node & 0xffff;
                    if (node < 0 || zn < z0 || zn >= z0 + TZ || xn < x0 || xn >= x0 + kTileX) {
                        raise_status(p.status, DUFWI_ERR_GEOMETRY);
                        continue;
                    }
                    p.cd[(static_cast<long long>(s) * p.nt + step) * p.n_rx + r] =
                        box[(zn - z0 + kHalo) * kBoxX + (xn - x0 + kHalo)];
                }
            }
        }
        // publish: every thread's stores and shared-memory reads are done before the release
        __syncthreads();
        // release by a thread of warp 1 (cumulative over the CTA's stores ordered by the barrier), so
        // that thread 0 can go on to the next item's counter wait and loads meanwhile
        if (tid == 32) st_release(sp.flags + k, i + 1);
    }
}

// ---- two time steps per launch ----------------------------------------------------------------
// Core tile 64 x 32 per CTA, 192 threads. Phase A computes U^{n+1} on the core plus a 4-cell
// ring (72 x 40, 180 blocks of 4 x 4) from an 80 x 48 TMA box of U^n and the 72 x 40 boxes of
// U^{n-1} and kappa'. Phase B computes U^{n+2} on the core (128 blocks) while the other two
// warps write the core of U^{n+1} and record receivers. Neighbouring CTAs read both input
// fields, so the outputs go to two other buffers (four rotating buffers per sweep). The
// adjoint runs the same two steps on mu (mu^m, then mu^{m-1}) with imaging of both.
constexpr int kPairZ = 32;
constexpr int kPairThreads = 192;
constexpr int kPairBoxX = kTileX + 4 * kHalo;    // 80
constexpr int kPairBoxZ = kPairZ + 4 * kHalo;    // 48
constexpr int kPairEX = kTileX + 2 * kHalo;      // 72
constexpr int kPairEZ = kPairZ + 2 * kHalo;      // 40

template <int MODE>
struct PairLayout {
    static constexpr int kBox = kPairBoxX * kPairBoxZ;
    static constexpr int kE = kPairEX * kPairEZ;
    static constexpr int kCore = kTileX * kPairZ;
    // box | prev (E) | kappa (E) | U^{n+1} (E) [| hist A | hist B | sums (core)]
    static constexpr int kLoadFloats = kBox + 2 * kE + (MODE == kAdjoint ? 3 * kCore : 0);
    static constexpr uint32_t kLoadBytes = kLoadFloats * sizeof(float);
    static constexpr int kFloats = kLoadFloats + kE;
    static constexpr uint32_t kBytes = kFloats * sizeof(float);
};

// Minimum resident CTAs of the two-step kernel per SM requested from the register allocator.
#ifndef DUFWI_STEP2_MIN_CTAS
#define DUFWI_STEP2_MIN_CTAS 3
#endif

template <int R, int MODE>
__global__ void __launch_bounds__(kPairThreads, DUFWI_STEP2_MIN_CTAS)
step2_kernel(const __grid_constant__ StepMaps tm, const StepParams p)
{
    using PL = PairLayout<MODE>;
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;
    __shared__ InjList inj[2];

    const int tid = threadIdx.x;
    const int s = p.shot0 + blockIdx.z;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * kPairZ;
    const int tx_idx = s % p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *box = smem;                       // U^n, origin (x0 - 8, z0 - 8)
    float *pe = box + PL::kBox;              // U^{n-1} on E, origin (x0 - 4, z0 - 4)
    float *ke = pe + PL::kE;                 // kappa' on E
    float *ha = ke + PL::kE;                 // adjoint: Lap(U^{m-1}) on the core
    float *hb = ha + PL::kCore;              // adjoint: Lap(U^{m-2}) on the core
    float *gs = hb + PL::kCore;              // adjoint: running imaging sums on the core
    float *n1 = smem + PL::kLoadFloats;      // U^{n+1} on E (computed)

    if (tid == 0) {
        prefetch_tensormap(&tm.cur_box);
        prefetch_tensormap(&tm.out_tile);
        mbar_init(&bar, 1);
    }
    __syncthreads();

    grid_dependency_wait();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, PL::kLoadBytes);
        tma_load_3d(box, &tm.cur_box, &bar, x0 - 2 * kHalo, z0 - 2 * kHalo, s);
        tma_load_3d(pe, &tm.out_tile, &bar, x0 - kHalo, z0 - kHalo, s);
        tma_load_3d(ke, &tm.kap_tile, &bar, x0 - kHalo, z0 - kHalo, s / p.n_tx);
        if (MODE == kAdjoint) {
            tma_load_4d(ha, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot);
            tma_load_4d(hb, &tm.hist_tile, &bar, x0, z0, s, p.hist_slot2);
            tma_load_3d(gs, &tm.grad_tile, &bar, x0, z0, s);
        }
    }
    grid_dependents_launch();

    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int n_tiles = gridDim.x * gridDim.y;
    int2 rx_core = make_int2(0, 0), rx_ring = make_int2(0, 0);
    if (MODE != kFwdHist) rx_core = __ldg(p.rx_tab + tx_idx * n_tiles + tile);
    if (MODE == kAdjoint) rx_ring = __ldg(p.rxe_tab + tx_idx * n_tiles + tile);
    // step A injections land anywhere on E, step B injections on the core
    const int step_b = MODE == kAdjoint ? p.step - 1 : p.step + 1;
    gather_injections<MODE>(inj[0], p, p.rxe_sorted, p.n_rxe, s, tx_idx, p.step, rx_ring, x0 - kHalo, z0 - kHalo,
                            kPairEX, kPairEZ, kPairEX, tid, kPairThreads);
    gather_injections<MODE>(inj[1], p, p.rx_sorted, p.n_rx, s, tx_idx, step_b, rx_core, x0, z0, kTileX, kPairZ,
                            kTileX, tid, kPairThreads);

    if (!wait_tile(&bar, p, tid)) return;

    // ---- phase A: step n -> n+1 on E (18 x 10 blocks)
    if (tid < 180) {
        const int ex = (tid % 18) * 4, ez = (tid / 18) * 4;             // E-local block origin
        const int gx = x0 - kHalo + ex;
        const bool interior = region_interior(p, map_grid(p, 0), x0 - kHalo, z0 - kHalo, kPairEX, kPairEZ);
        int xd[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, p.Nx);
        float4 lap[4], ctr[4];
        lap_block<R, kPairBoxX>(box, ex + kHalo, ez + kHalo, p.c, lap, ctr);
        const bool in_core = ex >= kHalo && ex < kHalo + kTileX && ez >= kHalo && ez < kHalo + kPairZ;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int lo = (ez + j) * kPairEX + ex;
            const int gz = z0 - kHalo + ez + j;
            const float4 v = eq2_row(ctr[j], ld4s(pe + lo), ld4s(ke + lo), lap[j], interior,
                                     p.damp_tab + layer_depth(gz, p.P, p.Nz) * (p.P + 1), xd);
            st4s(n1 + lo, v);
            if ((MODE == kFwdSampleHist || MODE == kFwdHist) && in_core && gz < p.nzp && gx < p.nxp) {
                float4 lv = lap[j];
                if (gx + 4 > p.nxp) {
                    if (gx + 1 >= p.nxp) lv.y = 0.f;
                    if (gx + 2 >= p.nxp) lv.z = 0.f;
                    lv.w = 0.f;
                }
                st4(p.hist + shot_off + static_cast<long long>(gz) * p.pitch + gx, lv);
            }
        }
    }
    __syncthreads();
    if (inj[0].n > 0) {
        if (tid == 0)
            apply_injections<MODE>(inj[0], n1, p, p.rxe_sorted, p.n_rxe, s, tx_idx, p.step, rx_ring, x0 - kHalo,
                                   z0 - kHalo, kPairEX, kPairEZ, kPairEX);
        __syncthreads();
    }

    // ---- phase B: step n+1 -> n+2 on the core (16 x 8 blocks); warps 4-5 write U^{n+1}
    float4 nxt[4], lap[4];
    const int lx = (tid & 15) * 4, lz = ((tid >> 4) & 7) * 4;
    const int gx = x0 + lx;
    if (tid < 128) {
        const bool interior = region_interior(p, map_grid(p, 0), x0, z0, kTileX, kPairZ);
        int xd[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, p.Nx);
        float4 ctr[4];
        lap_block<R, kPairEX>(n1, lx + kHalo, lz + kHalo, p.c, lap, ctr);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 prev = ld4s(box + (lz + j + 2 * kHalo) * kPairBoxX + lx + 2 * kHalo);
            const float4 kap = ld4s(ke + (lz + j + kHalo) * kPairEX + lx + kHalo);
            nxt[j] = eq2_row(ctr[j], prev, kap, lap[j], interior,
                             p.damp_tab + layer_depth(z0 + lz + j, p.P, p.Nz) * (p.P + 1), xd);
        }
    } else {
        // core of U^{n+1} (mu^m) to global, and receivers of U^n and U^{n+1}
        const int t = tid - 128;
        for (int k = t; k < kTileX / 4 * kPairZ; k += kPairThreads - 128) {
            const int cx = (k & 15) * 4, cz = k >> 4;
            const int gz = z0 + cz, gxx = x0 + cx;
            if (gz < p.nzp && gxx < p.nxp)
                st4(p.out + shot_off + static_cast<long long>(gz) * p.pitch + gxx,
                    ld4s(n1 + (cz + kHalo) * kPairEX + cx + kHalo));
        }
        if (MODE == kFwdSample || MODE == kFwdSampleHist) {
            const int cnt = (rx_core.x >= 0 && rx_core.y >= 0 && rx_core.x + rx_core.y <= p.n_rx) ? rx_core.y : 0;
            for (int e = t; e < cnt; e += kPairThreads - 128) {
                const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_core.x + e);
                const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
                const int zn = node >> 16, xn = node & 0xffff;
                if (node < 0 || zn < z0 || zn >= z0 + kPairZ || xn < x0 || xn >= x0 + kTileX) {
                    raise_status(p.status, DUFWI_ERR_GEOMETRY);
                    continue;
                }
                float *cd = p.cd + (static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r;
                cd[0] = box[(zn - z0 + 2 * kHalo) * kPairBoxX + (xn - x0 + 2 * kHalo)];
                if (p.step + 1 < p.nt) cd[p.n_rx] = n1[(zn - z0 + kHalo) * kPairEX + (xn - x0 + kHalo)];
            }
        }
    }
    if (inj[1].n > 0) {   // block-uniform: stage the core of U^{n+2} in the (free) U^{n-1} area
        __syncthreads();
        if (tid < 128) {
#pragma unroll
            for (int j = 0; j < 4; ++j) st4s(pe + (lz + j) * kTileX + lx, nxt[j]);
        }
        __syncthreads();
        if (tid == 0)
            apply_injections<MODE>(inj[1], pe, p, p.rx_sorted, p.n_rx, s, tx_idx, step_b, rx_core, x0, z0, kTileX,
                                   kPairZ, kTileX);
        __syncthreads();
        if (tid < 128) {
#pragma unroll
            for (int j = 0; j < 4; ++j) nxt[j] = ld4s(pe + (lz + j) * kTileX + lx);
        }
    }
    if (tid >= 128) return;

    const bool col_ok = gx < p.nxp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gz = z0 + lz + j;
        if (!col_ok || gz >= p.nzp) continue;
        float4 nv = nxt[j], lv = lap[j];
        if (gx + 4 > p.nxp) {
            if (gx + 1 >= p.nxp) { nv.y = 0.f; lv.y = 0.f; }
            if (gx + 2 >= p.nxp) { nv.z = 0.f; lv.z = 0.f; }
            nv.w = 0.f; lv.w = 0.f;
        }
        const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
        st4(p.out2 + o, nv);
        if (MODE == kFwdSampleHist || MODE == kFwdHist) st4(p.hist2 + o, lv);
        if (MODE == kAdjoint) {
            const int lo = (lz + j) * kTileX + lx;
            const float4 mu_m = ld4s(n1 + (lz + j + kHalo) * kPairEX + lx + kHalo);
            st4(p.grad + o, fma4(nv, ld4s(hb + lo), fma4(mu_m, ld4s(ha + lo), ld4s(gs + lo))));
        }
    }
}

// kappa' = C^2 (dt/dx)^2 / (1 + D dt) on the padded grid; C extended by edge replication.
// kappa' (and, with a density map, the half-point buoyancies) of one padded cell. Density and
// SoS are edge-replicated into the absorbing layer. With a density map the status word records
// non-finite or non-positive densities, and a local effective speed above c_max. That speed is
// C sqrt(g), with g the Gershgorin row sum of the symmetrised second-order density operator
// along each axis relative to its value in a uniform medium; g <= 1.21 at any density step, and
// the check guards the time step rather than proving stability.
__global__ void setup_kappa_kernel(const float *sos, const float *density, float *kap, float *bxo, float *bzo,
                                   int *status, int NxE, int NzE, int P, int nxpE, int nzpE, int pitch, double r2,
                                   double d0, double dt, double c_max, const int2 *map_dims, bool unit_b)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int b = blockIdx.z;
    if (x >= pitch) return;
    // grid of this map (sized calls: its own, inside the envelope slab [NzE][NxE] of the map)
    const int Nx = map_dims ? map_dims[b].x : NxE, Nz = map_dims ? map_dims[b].y : NzE;
    const int nxp = Nx + 2 * P, nzp = Nz + 2 * P;
    const long long o = (static_cast<long long>(b) * nzpE + z) * pitch + x;
    if (x >= nxp || z >= nzp) {
        kap[o] = 0.f;
        if (density || unit_b) { bxo[o] = 0.f; bzo[o] = 0.f; }
        return;
    }
    if (unit_b) {
        bxo[o] = x + 1 < nxp ? 1.f : 0.f;
        bzo[o] = z + 1 < nzp ? 1.f : 0.f;
    }
    auto src_of = [&](int xx, int zz) {
        const int xs = min(max(xx - P, 0), Nx - 1), zs = min(max(zz - P, 0), Nz - 1);
        return (static_cast<long long>(b) * NzE + zs) * NxE + xs;
    };
    const long long src = src_of(x, z);
    const double C = sos[src];
    double ceff = C, rho = 1.0;
    if (density) {
        rho = density[src];
        const bool interior_cell = x >= P && x < P + Nx && z >= P && z < P + Nz;
        if (interior_cell && !isfinite(rho)) raise_status(status, DUFWI_ERR_NONFINITE);
        else if (interior_cell && !(rho > 0.0)) raise_status(status, DUFWI_ERR_INVALID_ARG);
        const double rx = x + 1 < nxp ? static_cast<double>(density[src_of(x + 1, z)]) : rho;
        const double rz = z + 1 < nzp ? static_cast<double>(density[src_of(x, z + 1)]) : rho;
        const double rxm = x > 0 ? static_cast<double>(density[src_of(x - 1, z)]) : rho;
        const double rzm = z > 0 ? static_cast<double>(density[src_of(x, z - 1)]) : rho;
        bxo[o] = x + 1 < nxp ? static_cast<float>(2.0 / (rho + rx)) : 0.f;
        bzo[o] = z + 1 < nzp ? static_cast<float>(2.0 / (rho + rz)) : 0.f;
        auto row_sum = [rho](double rp, double rm) {
            const double bp = 2.0 / (rho + rp), bm = 2.0 / (rho + rm);
            return 0.25 * (rho * (bp + bm) + sqrt(rho * rp) * bp + sqrt(rho * rm) * bm);
        };
        ceff = C * sqrt(fmax(row_sum(rx, rxm), row_sum(rz, rzm)));
    }
    if (!isfinite(C)) raise_status(status, DUFWI_ERR_NONFINITE);
    else if (!(C > 0.0) || C > c_max || (density && ceff > c_max)) raise_status(status, DUFWI_ERR_CFL);
    const int dxl = x < P ? P - x : (x > P + Nx - 1 ? x - (P + Nx - 1) : 0);
    const int dzl = z < P ? P - z : (z > P + Nz - 1 ? z - (P + Nz - 1) : 0);
    const double xx = static_cast<double>(dxl) / P, zz = static_cast<double>(dzl) / P;
    const double D = d0 * xx * xx + d0 * zz * zz;
    kap[o] = static_cast<float>(rho * C * C * r2 / (1.0 + D * dt));
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
// kappa'_r * 2 (M_sim - M_obs). cd_lo (or null): low parts of M_sim from the compensated steps.
__global__ void residual_kernel(const float *cd_sim, const float *cd_lo, const float *cd_obs, const float *kap,
                                const int *rx_node, float *asrc, double *partial, int *status, int n_tx, int n_rx,
                                int nt, long long slice, int pitch)
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
        // with the compensated forward steps the traces are hi + lo: (hi - obs) is exact when the two
        // are within a factor 2 of each other, and lo then adds what the rounding of M_sim dropped
        float d = cd_sim[base + i] - obs;
        if (cd_lo) d += cd_lo[base + i];
        acc += static_cast<double>(d) * static_cast<double>(d);
        const int node = rx_node[tx_idx * n_rx + r];
        const float kr = kap[map * slice + static_cast<long long>(node >> 16) * pitch + (node & 0xffff)];
        asrc[base + i] = kr * (2.0f * d);
    }
    if (bad) raise_status(status, DUFWI_ERR_NONFINITE);
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) partial[s] = t;
}

// dkappa' = kappa' * 2 dC / C (kappa' = C^2 dt^2/(dx^2 (1 + D dt)) so dkappa'/dC = 2 kappa'/C),
// with C and dC extended into the absorbing layer by edge replication.
__global__ void setup_dkappa_kernel(const float *sos, const float *dsos, const float *kap, float *dkap, int Nx, int Nz,
                                    int P, int nzp, int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int b = blockIdx.z;
    if (x >= pitch) return;
    const long long o = (static_cast<long long>(b) * nzp + z) * pitch + x;
    const int xs = min(max(x - P, 0), Nx - 1), zs = min(max(z - P, 0), Nz - 1);
    const long long src = (static_cast<long long>(b) * Nz + zs) * Nx + xs;
    const double k = kap[o];   // zero on the pitch padding
    dkap[o] = static_cast<float>(k * 2.0 * static_cast<double>(dsos[src]) / static_cast<double>(sos[src]));
}

// Adjoint source of a general cotangent v = dL/dM: kappa'_r * v (no misfit).
__global__ void cotangent_source_kernel(const float *cd_grad, const float *kap, const int *rx_node, float *asrc,
                                        int *status, int n_tx, int n_rx, int nt, long long slice, int pitch)
{
    const int s = blockIdx.y;
    const int tx_idx = s % n_tx, map = s / n_tx;
    const long long base = static_cast<long long>(s) * nt * n_rx;
    const long long n = static_cast<long long>(nt) * n_rx;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(i % n_rx);
        const float v = cd_grad[base + i];
        if (!isfinite(v)) raise_status(status, DUFWI_ERR_NONFINITE);
        const int node = rx_node[tx_idx * n_rx + r];
        asrc[base + i] = kap[map * slice + static_cast<long long>(node >> 16) * pitch + (node & 0xffff)] * v;
    }
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
__global__ void fold_x_kernel(const float *g_shot, double *fx, int n_tx, int NxE, int P, int nzpE, long long slice,
                              int pitch, const int2 *map_dims)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int zp = blockIdx.y;
    const int b = blockIdx.z;
    const int Nx = map_dims ? map_dims[b].x : NxE;
    if (ix >= Nx) return;
    const int xlo = ix == 0 ? 0 : ix + P, xhi = ix == Nx - 1 ? Nx + 2 * P - 1 : ix + P;
    double acc = 0.0;
    for (int t = 0; t < n_tx; ++t) {
        const float *g = g_shot + static_cast<long long>(b * n_tx + t) * slice + static_cast<long long>(zp) * pitch;
        for (int x = xlo; x <= xhi; ++x) acc += g[x];
    }
    fx[(static_cast<long long>(b) * nzpE + zp) * NxE + ix] = acc;
}

template <typename T>
__global__ void fold_z_kernel(const double *fx, const float *sos, T *grad, int NxE, int NzE, int P, int nzpE,
                              const int2 *map_dims)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int b = blockIdx.z;
    if (ix >= NxE) return;
    const int Nx = map_dims ? map_dims[b].x : NxE, Nz = map_dims ? map_dims[b].y : NzE;
    const long long o = (static_cast<long long>(b) * NzE + iz) * NxE + ix;
    if (ix >= Nx || iz >= Nz) { grad[o] = T(0); return; }   // outside this map (sized calls)
    const int zlo = iz == 0 ? 0 : iz + P, zhi = iz == Nz - 1 ? Nz + 2 * P - 1 : iz + P;
    double acc = 0.0;
    for (int z = zlo; z <= zhi; ++z) acc += fx[(static_cast<long long>(b) * nzpE + z) * NxE + ix];
    grad[o] = static_cast<T>(acc * (2.0 / static_cast<double>(sos[o])));
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

// <one-step kernel source>
template <int R, int MODE, int TZ, int MINB = 0>
static cudaError_t launch_step_rmt(const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    using TL = TileLayout<MODE, TZ>;
    static DeviceCache dc;   // shared-memory attributes, set once per device
    cudaError_t e = configure_kernel(step_kernel<R, MODE, TZ, MINB>, TL::kBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + TZ - 1) / TZ, p.n_shots);
    cfg.blockDim = dim3(TL::kThreadsPerCta);
    cfg.dynamicSmemBytes = TL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step_kernel<R, MODE, TZ, MINB>, tm, p);
}

template <int R, int MODE>
static cudaError_t launch_step_rm(const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    if constexpr (R == 4) {   // register-cap variants of the 64 x 32 form (p.min_ctas; 0 = default)
        if (p.tile_z == 32 && p.min_ctas == 4) return launch_step_rmt<R, MODE, 32, 4>(tm, p, st);
        if (p.tile_z == 32 && p.min_ctas == 6) return launch_step_rmt<R, MODE, 32, 6>(tm, p, st);
    }
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
    case kBorn: return launch_step_rm<R, kBorn>(tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R, int MODE>
static cudaError_t launch_step_mt_rm(const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    using TL = TileLayout<MODE, 32>;
    constexpr uint32_t kBytes = 2 * TL::kBytes;   // two stages
    static DeviceCache dc;
    int resident = 0;
    cudaError_t e = resident_ctas(step_mt_kernel<R, MODE>, TL::kThreadsPerCta, kBytes, dc, &resident);
    if (e != cudaSuccess) return e;
    const long long tiles = static_cast<long long>((p.nxp + kTileX - 1) / kTileX) * ((p.nzp + 31) / 32) *
                            p.n_maps * p.n_tx;
    if (tiles >= (1ll << 31)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(std::min<long long>(tiles, resident)));
    cfg.blockDim = dim3(TL::kThreadsPerCta);
    cfg.dynamicSmemBytes = kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step_mt_kernel<R, MODE>, tm, p);
}

template <int R>
static cudaError_t launch_step_mt_r(int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_step_mt_rm<R, kFwdSample>(tm, p, st);
    case kFwdSampleHist: return launch_step_mt_rm<R, kFwdSampleHist>(tm, p, st);
    case kFwdHist: return launch_step_mt_rm<R, kFwdHist>(tm, p, st);
    case kAdjoint: return launch_step_mt_rm<R, kAdjoint>(tm, p, st);
    case kBorn: return launch_step_mt_rm<R, kBorn>(tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

// </one-step kernel source>

template <int R, int MODE>
static cudaError_t launch_step2_rm(const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    using PL = PairLayout<MODE>;
    static DeviceCache dc;   // shared-memory attributes, set once per device
    cudaError_t e = configure_kernel(step2_kernel<R, MODE>, PL::kBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + kPairZ - 1) / kPairZ, p.n_shots);
    cfg.blockDim = dim3(kPairThreads);
    cfg.dynamicSmemBytes = PL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step2_kernel<R, MODE>, tm, p);
}

template <int R>
static cudaError_t launch_step2_r(int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_step2_rm<R, kFwdSample>(tm, p, st);
    case kFwdSampleHist: return launch_step2_rm<R, kFwdSampleHist>(tm, p, st);
    case kFwdHist: return launch_step2_rm<R, kFwdHist>(tm, p, st);
    case kAdjoint: return launch_step2_rm<R, kAdjoint>(tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step2(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    switch (radius) {
    case 1: return launch_step2_r<1>(mode, tm, p, st);
    case 2: return launch_step2_r<2>(mode, tm, p, st);
    case 3: return launch_step2_r<3>(mode, tm, p, st);
    case 4: return launch_step2_r<4>(mode, tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R, int MODE>
static cudaError_t launch_sweep_rm(const SweepMaps &tm, const StepParams &p, const SweepParams &sp, int *grid_ctas,
                                   cudaStream_t st)
{
    using TL = TileLayout<MODE, 32>;
    static DeviceCache dc;   // attributes and co-resident CTAs of this variant, per device
    int max_ctas = 0;
    cudaError_t e = resident_ctas(sweep_kernel<R, MODE>, 128, TL::kBytes, dc, &max_ctas);
    if (e != cudaSuccess) return e;
    const long long items = static_cast<long long>(sp.n_steps) * sp.tiles;
    if (items >= (1ll << 31)) return cudaErrorInvalidValue;
    // Items of one round (grid consecutive items) must not depend on each other, or the round
    // serialises: dependencies lie tiles - tiles_x items back at the least.
    const int no_chain = std::max(1, sp.tiles - sp.tiles_x);
    const int grid = static_cast<int>(std::min<long long>(std::min<long long>(items, max_ctas), no_chain));
    if (grid_ctas) *grid_ctas = grid;
    if (grid < 1) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = TL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sweep_kernel<R, MODE>, tm, p, sp);
}

template <int R>
static cudaError_t launch_sweep_r(int mode, const SweepMaps &tm, const StepParams &p, const SweepParams &sp,
                                  int *grid_ctas, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_sweep_rm<R, kFwdSample>(tm, p, sp, grid_ctas, st);
    case kFwdSampleHist: return launch_sweep_rm<R, kFwdSampleHist>(tm, p, sp, grid_ctas, st);
    case kFwdHist: return launch_sweep_rm<R, kFwdHist>(tm, p, sp, grid_ctas, st);
    case kAdjoint: return launch_sweep_rm<R, kAdjoint>(tm, p, sp, grid_ctas, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep(int radius, int mode, const SweepMaps &tm, const StepParams &p, const SweepParams &sp,
                         int *grid_ctas, cudaStream_t st)
{
    if (p.tile_z != 32) return cudaErrorInvalidValue;
    switch (radius) {
    case 1: return launch_sweep_r<1>(mode, tm, p, sp, grid_ctas, st);
    case 2: return launch_sweep_r<2>(mode, tm, p, sp, grid_ctas, st);
    case 3: return launch_sweep_r<3>(mode, tm, p, sp, grid_ctas, st);
    case 4: return launch_sweep_r<4>(mode, tm, p, sp, grid_ctas, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R, int MODE>
static cudaError_t launch_step_cpml_rm(const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                                       const CpmlParams &cp, cudaStream_t st)
{
    using CL = CpmlLayout<MODE>;
    static DeviceCache dc;   // shared-memory attributes, set once per device
    cudaError_t e = configure_kernel(cpml_step_kernel<R, MODE, 0>, CL::kBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + kVTileZ - 1) / kVTileZ, p.n_shots);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = CL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SoParams q;
    memset(&q, 0, sizeof(q));
    return cudaLaunchKernelEx(&cfg, cpml_step_kernel<R, MODE, 0>, tm, cm, p, cp, q);
}

template <int R, int KIND>
static cudaError_t launch_so_step_cpml_rk(const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                                          const CpmlParams &cp, const SoParams &q, cudaStream_t st)
{
    constexpr int MODE = KIND == kSoBorn ? kFwdHist : kAdjoint;
    using CL = CpmlLayout<MODE, 1 + KIND>;
    static DeviceCache dc;   // shared-memory attributes, set once per device
    cudaError_t e = configure_kernel(cpml_step_kernel<R, MODE, 1 + KIND>, CL::kBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + kVTileZ - 1) / kVTileZ, p.n_shots);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = CL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cpml_step_kernel<R, MODE, 1 + KIND>, tm, cm, p, cp, q);
}

template <int R>
static cudaError_t launch_so_step_cpml_r(int kind, const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                                         const CpmlParams &cp, const SoParams &q, cudaStream_t st)
{
    switch (kind) {
    case kSoBorn: return launch_so_step_cpml_rk<R, kSoBorn>(tm, cm, p, cp, q, st);
    case kSoAdj: return launch_so_step_cpml_rk<R, kSoAdj>(tm, cm, p, cp, q, st);
    case kSoBornAdj: return launch_so_step_cpml_rk<R, kSoBornAdj>(tm, cm, p, cp, q, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_so_step_cpml(int radius, int kind, const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                                const CpmlParams &cp, const SoParams &q, cudaStream_t st)
{
    if (p.tile_z != kVTileZ || p.map_dims || p.tile_class != 2) return cudaErrorInvalidValue;
    switch (radius) {
    case 1: return launch_so_step_cpml_r<1>(kind, tm, cm, p, cp, q, st);
    case 2: return launch_so_step_cpml_r<2>(kind, tm, cm, p, cp, q, st);
    case 3: return launch_so_step_cpml_r<3>(kind, tm, cm, p, cp, q, st);
    case 4: return launch_so_step_cpml_r<4>(kind, tm, cm, p, cp, q, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R>
static cudaError_t launch_step_cpml_r(int mode, const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                                      const CpmlParams &cp, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_step_cpml_rm<R, kFwdSample>(tm, cm, p, cp, st);
    case kFwdSampleHist: return launch_step_cpml_rm<R, kFwdSampleHist>(tm, cm, p, cp, st);
    case kFwdHist: return launch_step_cpml_rm<R, kFwdHist>(tm, cm, p, cp, st);
    case kAdjoint: return launch_step_cpml_rm<R, kAdjoint>(tm, cm, p, cp, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_cpml(int radius, int mode, const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                             const CpmlParams &cp, cudaStream_t st)
{
    if (p.tile_z != kVTileZ || p.map_dims) return cudaErrorInvalidValue;
    switch (radius) {
    case 1: return launch_step_cpml_r<1>(mode, tm, cm, p, cp, st);
    case 2: return launch_step_cpml_r<2>(mode, tm, cm, p, cp, st);
    case 3: return launch_step_cpml_r<3>(mode, tm, cm, p, cp, st);
    case 4: return launch_step_cpml_r<4>(mode, tm, cm, p, cp, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R, int MODE>
static cudaError_t launch_step_vd_rm(const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    using VL = VdLayout<MODE>;
    static DeviceCache dc;   // shared-memory attributes, set once per device
    cudaError_t e = configure_kernel(vd_step_kernel<R, MODE>, VL::kBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + kVTileZ - 1) / kVTileZ, p.n_shots);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = VL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, vd_step_kernel<R, MODE>, tm, p);
}

template <int R>
static cudaError_t launch_step_vd_r(int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_step_vd_rm<R, kFwdSample>(tm, p, st);
    case kFwdSampleHist: return launch_step_vd_rm<R, kFwdSampleHist>(tm, p, st);
    case kFwdHist: return launch_step_vd_rm<R, kFwdHist>(tm, p, st);
    case kAdjoint: return launch_step_vd_rm<R, kAdjoint>(tm, p, st);
    case kBorn: return launch_step_vd_rm<R, kBorn>(tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_vd(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    if (p.tile_z != kVTileZ) return cudaErrorInvalidValue;
    switch (radius) {
    case 1: return launch_step_vd_r<1>(mode, tm, p, st);
    case 2: return launch_step_vd_r<2>(mode, tm, p, st);
    case 3: return launch_step_vd_r<3>(mode, tm, p, st);
    case 4: return launch_step_vd_r<4>(mode, tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R, int KIND, bool VD>
static cudaError_t launch_so_step_rk(const SoMaps &tm, const StepParams &p, const SoParams &q, cudaStream_t st)
{
    using SL = SoLayout<KIND, VD>;
    static DeviceCache dc;   // shared-memory attributes, set once per device
    cudaError_t e = configure_kernel(so_step_kernel<R, KIND, VD>, SL::kBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + 31) / 32, p.n_shots);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = SL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, so_step_kernel<R, KIND, VD>, tm, p, q);
}

template <int R, bool VD>
static cudaError_t launch_so_step_r(int kind, const SoMaps &tm, const StepParams &p, const SoParams &q,
                                    cudaStream_t st)
{
    switch (kind) {
    case kSoBorn: return launch_so_step_rk<R, kSoBorn, VD>(tm, p, q, st);
    case kSoAdj: return launch_so_step_rk<R, kSoAdj, VD>(tm, p, q, st);
    case kSoBornAdj: return launch_so_step_rk<R, kSoBornAdj, VD>(tm, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

template <bool VD>
static cudaError_t launch_so_step_v(int radius, int kind, const SoMaps &tm, const StepParams &p, const SoParams &q,
                                    cudaStream_t st)
{
    switch (radius) {
    case 1: return launch_so_step_r<1, VD>(kind, tm, p, q, st);
    case 2: return launch_so_step_r<2, VD>(kind, tm, p, q, st);
    case 3: return launch_so_step_r<3, VD>(kind, tm, p, q, st);
    case 4: return launch_so_step_r<4, VD>(kind, tm, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_so_step(int radius, int kind, bool vd, const SoMaps &tm, const StepParams &p, const SoParams &q,
                           cudaStream_t st)
{
    if (p.tile_z != 32 || p.map_dims) return cudaErrorInvalidValue;
    return vd ? launch_so_step_v<true>(radius, kind, tm, p, q, st) : launch_so_step_v<false>(radius, kind, tm, p, q, st);
}

cudaError_t launch_hvp_source(const float *cd_sim, const float *cd_obs, const float *dcd, const float *kap,
                              const float *dkap, const int *rx_node, float *asrc2, int S, int n_tx, int n_rx, int nt,
                              long long slice, int pitch, cudaStream_t st)
{
    if (n_rx == 0) return cudaSuccess;
    const long long n = static_cast<long long>(nt) * n_rx;
    dim3 grid(static_cast<unsigned>(std::min<long long>((n + 255) / 256, 64)), S);
    hvp_source_kernel<<<grid, 256, 0, st>>>(cd_sim, cd_obs, dcd, kap, dkap, rx_node, asrc2, n_tx, n_rx, nt, slice,
                                            pitch);
    return cudaGetLastError();
}

cudaError_t launch_so_combine(float *a, const float *b, const float *g, const float *sos, const float *dsos, int S,
                              int n_tx, int Nx, int Nz, int P, int nzp, int pitch, long long slice, cudaStream_t st)
{
    so_combine_kernel<<<dim3((pitch + 127) / 128, nzp, S), 128, 0, st>>>(a, b, g, sos, dsos, n_tx, Nx, Nz, P, pitch,
                                                                          slice);
    return cudaGetLastError();
}

// <one-step kernel source>
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

cudaError_t launch_step_mt(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st)
{
    if (p.tile_z != 32) return cudaErrorInvalidValue;
    switch (radius) {
    case 1: return launch_step_mt_r<1>(mode, tm, p, st);
    case 2: return launch_step_mt_r<2>(mode, tm, p, st);
    case 3: return launch_step_mt_r<3>(mode, tm, p, st);
    case 4: return launch_step_mt_r<4>(mode, tm, p, st);
    default: return cudaErrorInvalidValue;
    }
}

// </one-step kernel source>

// Dynamic shared memory of the cluster form at most (the kernel's static lists take about 2 KB
// of the 227 KB a CTA may use).
constexpr size_t kClusterSmemMax = 220 * 1024;

size_t cluster_smem_bytes(int nxp, int nzp, int *H, int *lpitch)
{
    const int h = ((nzp + kClusterCtas - 1) / kClusterCtas + 3) / 4 * 4;
    const int lp = (nxp + 3) / 4 * 4 + 8;
    const size_t bytes = (size_t)(3 * (h + 8) + 2 * h) * lp * sizeof(float);
    if (H) *H = h;
    if (lpitch) *lpitch = lp;
    return bytes <= (size_t)kClusterSmemMax ? bytes : 0;
}

template <int R, int MODE>
static cudaError_t launch_cluster_sweep_rm(const StepParams &p, const ClusterParams &cp, cudaStream_t st)
{
    int H = 0, lp = 0;
    const size_t bytes = cluster_smem_bytes(p.nxp, p.nzp, &H, &lp);
    if (bytes == 0 || H != cp.H || lp != cp.lpitch || p.map_dims) return cudaErrorInvalidValue;
    static DeviceCache dc;   // shared-memory attributes, set once per device (to the largest size used)
    cudaError_t e = configure_kernel(cluster_sweep_kernel<R, MODE>, (uint32_t)kClusterSmemMax, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas, p.n_shots);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_sweep_kernel<R, MODE>, p, cp);
}

template <int R>
static cudaError_t launch_cluster_sweep_r(int mode, const StepParams &p, const ClusterParams &cp, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_cluster_sweep_rm<R, kFwdSample>(p, cp, st);
    case kFwdSampleHist: return launch_cluster_sweep_rm<R, kFwdSampleHist>(p, cp, st);
    case kFwdHist: return launch_cluster_sweep_rm<R, kFwdHist>(p, cp, st);
    case kAdjoint: return launch_cluster_sweep_rm<R, kAdjoint>(p, cp, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cluster_sweep(int radius, int mode, const StepParams &p, const ClusterParams &cp, cudaStream_t st)
{
    switch (radius) {
    case 1: return launch_cluster_sweep_r<1>(mode, p, cp, st);
    case 2: return launch_cluster_sweep_r<2>(mode, p, cp, st);
    case 3: return launch_cluster_sweep_r<3>(mode, p, cp, st);
    case 4: return launch_cluster_sweep_r<4>(mode, p, cp, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_setup_kappa(const float *sos, const float *density, float *kap, float *bx, float *bz, int *status,
                               int n_maps, int Nx, int Nz, int P, int nxp, int nzp, int pitch, double dt_over_dx,
                               double d0, double dt, double c_max, const int2 *map_dims, bool unit_b,
                               cudaStream_t st)
{
    if ((density || unit_b) && (!bx || !bz)) return cudaErrorInvalidValue;
    dim3 grid((pitch + 127) / 128, nzp, n_maps);
    setup_kappa_kernel<<<grid, 128, 0, st>>>(sos, density, kap, bx, bz, status, Nx, Nz, P, nxp, nzp, pitch,
                                             dt_over_dx * dt_over_dx, d0, dt, c_max, map_dims, unit_b);
    return cudaGetLastError();
}

cudaError_t launch_sample(const float *field, const int *rx_node, float *cd, long long slice, int pitch, int S,
                          int n_tx, int n_rx, int nt, int step, cudaStream_t st)
{
    if (n_rx == 0) return cudaSuccess;
    sample_kernel<<<S, 128, 0, st>>>(field, rx_node, cd, slice, pitch, n_tx, n_rx, nt, step);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float *cd_sim, const float *cd_lo, const float *cd_obs, const float *kap,
                            const int *rx_node, float *asrc, double *partial, int *status, int S, int n_tx, int n_rx,
                            int nt, long long slice, int pitch, cudaStream_t st)
{
    residual_kernel<<<S, 512, 0, st>>>(cd_sim, cd_lo, cd_obs, kap, rx_node, asrc, partial, status, n_tx, n_rx, nt,
                                       slice, pitch);
    return cudaGetLastError();
}

cudaError_t launch_setup_dkappa(const float *sos, const float *dsos, const float *kap, float *dkap, int n_maps, int Nx,
                                int Nz, int P, int nzp, int pitch, cudaStream_t st)
{
    setup_dkappa_kernel<<<dim3((pitch + 127) / 128, nzp, n_maps), 128, 0, st>>>(sos, dsos, kap, dkap, Nx, Nz, P, nzp,
                                                                                pitch);
    return cudaGetLastError();
}

cudaError_t launch_cotangent_source(const float *cd_grad, const float *kap, const int *rx_node, float *asrc,
                                   int *status, int S, int n_tx, int n_rx, int nt, long long slice, int pitch,
                                   cudaStream_t st)
{
    if (n_rx == 0) return cudaSuccess;
    const long long n = static_cast<long long>(nt) * n_rx;
    dim3 grid(static_cast<unsigned>(std::min<long long>((n + 255) / 256, 64)), S);
    cotangent_source_kernel<<<grid, 256, 0, st>>>(cd_grad, kap, rx_node, asrc, status, n_tx, n_rx, nt, slice, pitch);
    return cudaGetLastError();
}

cudaError_t launch_misfit_sum(const double *partial, double *misfit, int n_maps, int n_tx, cudaStream_t st)
{
    misfit_sum_kernel<<<(n_maps + 127) / 128, 128, 0, st>>>(partial, misfit, n_maps, n_tx);
    return cudaGetLastError();
}

cudaError_t launch_fold(const float *g_shot, const float *sos, float *grad, double *grad64, double *fx, int n_maps,
                        int n_tx, int Nx, int Nz, int P, long long slice, int pitch, const int2 *map_dims,
                        cudaStream_t st)
{
    const int nzp = Nz + 2 * P;
    fold_x_kernel<<<dim3((Nx + 127) / 128, nzp, n_maps), 128, 0, st>>>(g_shot, fx, n_tx, Nx, P, nzp, slice, pitch,
                                                                       map_dims);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (grad64)
        fold_z_kernel<double><<<dim3((Nx + 127) / 128, Nz, n_maps), 128, 0, st>>>(fx, sos, grad64, Nx, Nz, P, nzp,
                                                                                   map_dims);
    else
        fold_z_kernel<float><<<dim3((Nx + 127) / 128, Nz, n_maps), 128, 0, st>>>(fx, sos, grad, Nx, Nz, P, nzp,
                                                                                 map_dims);
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
