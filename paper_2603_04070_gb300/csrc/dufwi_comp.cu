// dufwi_comp.cu -- compensated forward step of Eq. 2: the field is carried as an unevaluated sum
// of two FP32 numbers (hi + lo, "double-float"), and every rounding of the step is recovered with
// error-free transformations, so that the simulated traces keep about 44 bits.
//
// Why: the misfit gradient (Eq. 6) is linear in the residual M_sim - M_obs. When the scatterer is
// weak, that residual is a small part of the traces (0.1-2 % on the 128 x 128 disk workload), and
// any rounding of the simulated traces enters the gradient amplified by |M| / |r|. A plain FP32
// step leaves a trace error of ~1e-6 and gradient errors of 1e-3 to 1e-2 there; rounding the exact
// traces to FP32 once is already worth up to 4e-4. With this step the trace error is that of the
// FP64 recursion (~1e-13), and the residual is formed from (hi, lo) before any rounding.
//
// The step, in exact arithmetic the one of the plain kernel:
//   U^{n+1} = 2 U^n - U^{n-1} + [(a - 2) U^n + (b + 1) U^{n-1}] + kq S(U^n) + s^n
// with S the central stencil with integer weights c'_k = s_R c_k (the textbook weights times the
// least common multiple of their denominators: s_R = 1, 12, 180, 5040 for orders 2 to 8; S sums
// them exactly up to the tracked roundings), and kq = kappa' / s_R. The coefficients kq (per cell)
// and (a - 2), (b + 1) (per pair of layer depths) are FP64 values split into hi + lo on the host or
// in the setup kernel, so no coefficient is rounded to FP32 either: a rounded coefficient is a
// systematic perturbation of the medium or of the layer, which the traces see coherently.
//
// Arithmetic per cell: S(U_hi) with TwoSum / TwoProd on every operation (the error terms summed
// in FP32), S(U_lo) in plain FP32 (its rounding is relative to |U_lo| ~ 2^-24 |U|), the update in
// double-float, and a final TwoSum that renormalises (hi, lo). Operations use the round-to-nearest
// intrinsics, which the compiler neither contracts nor reorders.
//
// Tile scheme: 64 x 32 output tiles of one shot, 128 threads, a 4 (x) x 4 (z) block per thread;
// one mbarrier collects the TMA loads of the 72 x 40 boxes of U_hi^n and U_lo^n, and of the 64 x 32
// tiles of U_hi^{n-1}, U_lo^{n-1}, kq_hi and kq_lo. Both planes of U^{n+1} are written in place of
// U^{n-1}. The channel data are sampled as (hi, lo) from the boxes; the history (Lap U^n with the
// textbook weights, for the imaging condition) is written rounded to FP32.
#include "dufwi_internal.h"

#include "../../include/dufwi.h"
#include "dufwi_device.cuh"

namespace dufwi {
namespace {

constexpr int kCompTileZ = 32;
constexpr int kCompBoxRows = kCompTileZ + 2 * kHalo;
constexpr int kCompBox = kBoxX * kCompBoxRows;          // 72 x 40
constexpr int kCompTile = kTileX * kCompTileZ;          // 64 x 32
constexpr uint32_t kCompBytes = (2 * kCompBox + 4 * kCompTile) * sizeof(float);

// Integer weights c'_k = s_R c_k of the central stencil of radius R (k = 1..R; the centre weight
// is -2 sum_k c'_k per axis, applied through the difference form).
template <int R>
__device__ __forceinline__ float int_weight(int k)
{
    if (R == 1) return 1.0f;
    if (R == 2) return k == 1 ? 16.0f : -1.0f;
    if (R == 3) return k == 1 ? 270.0f : (k == 2 ? -27.0f : 2.0f);
    return k == 1 ? 8064.0f : (k == 2 ? -1008.0f : (k == 3 ? 128.0f : -9.0f));
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// s + e = a + b exactly (Knuth's TwoSum; any magnitudes), two lanes at a time.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
}

// p + e = a * b exactly (the FMA gives the rounding error of the product).
__device__ __forceinline__ void two_prod2(float2 a, float2 b, float2 &p, float2 &e)
{
    p = __fmul2_rn(a, b);
    e = __ffma2_rn(a, b, neg2(p));
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float2 lane2(float4 v, int h) { return h == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w); }

// Stencil S of one row of four cells (two packed pairs h = 0, 1) of a shared-memory plane with
// row stride kBoxX, centre at (cx, cz) of the box. compensated: S(hi) as (sum, error) pairs;
// otherwise the plain FP32 sum (error left untouched).
template <int R, bool COMP>
__device__ __forceinline__ void stencil_row(const float *src, int cx, int cz, float2 (&sum)[2], float2 (&err)[2])
{
    const float4 lft = ld4s(src + cz * kBoxX + cx - 4);
    const float4 ctr = ld4s(src + cz * kBoxX + cx);
    const float4 rgt = ld4s(src + cz * kBoxX + cx + 4);
    const float w[12] = {lft.x, lft.y, lft.z, lft.w, ctr.x, ctr.y, ctr.z, ctr.w, rgt.x, rgt.y, rgt.z, rgt.w};
    float4 zm[R], zp[R];
#pragma unroll
    for (int k = 1; k <= R; ++k) {
        zm[k - 1] = ld4s(src + (cz - k) * kBoxX + cx);
        zp[k - 1] = ld4s(src + (cz + k) * kBoxX + cx);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 u = make_float2(w[4 + 2 * h], w[5 + 2 * h]);
        const float2 m4 = __fmul2_rn(make_float2(-4.0f, -4.0f), u);   // exact
        float2 acc = make_float2(0.f, 0.f), e = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            const float2 cw = make_float2(int_weight<R>(k), int_weight<R>(k));
            const float2 xm = make_float2(w[4 + 2 * h - k], w[5 + 2 * h - k]);
            const float2 xp = make_float2(w[4 + 2 * h + k], w[5 + 2 * h + k]);
            const float2 zmv = lane2(zm[k - 1], h), zpv = lane2(zp[k - 1], h);
            if (COMP) {
                float2 xs, ex, zs, ez, t, et, q, eq, p, ep;
                two_sum2(xm, xp, xs, ex);
                two_sum2(zmv, zpv, zs, ez);
                two_sum2(xs, zs, t, et);
                two_sum2(t, m4, q, eq);
                two_prod2(cw, q, p, ep);
                const float2 ein = __fadd2_rn(__fadd2_rn(ex, ez), __fadd2_rn(et, eq));
                if (k == 1) {
                    acc = p;
                    e = __ffma2_rn(cw, ein, ep);
                } else {
                    float2 s, ea;
                    two_sum2(acc, p, s, ea);
                    acc = s;
                    e = __ffma2_rn(cw, ein, __fadd2_rn(e, __fadd2_rn(ep, ea)));
                }
            } else {
                const float2 t = __fadd2_rn(__fadd2_rn(__fadd2_rn(xm, xp), __fadd2_rn(zmv, zpv)), m4);
                acc = __ffma2_rn(cw, t, acc);
            }
        }
        sum[h] = acc;
        if (COMP) err[h] = e;
    }
}

__device__ __forceinline__ float4 f4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// Bounded wait of every thread on the CTA's load barrier (no thread parks behind another). On a
// timeout the status word records it, and the thread waits once more (bounded) so that copies
// still in flight land before the CTA exits.
__device__ __forceinline__ bool comp_wait(uint64_t *bar, const StepParams &p)
{
    if (mbar_wait_bounded(bar, 0)) return true;
    raise_status(p.status, DUFWI_ERR_TIMEOUT);
    mbar_wait_bounded(bar, 0);
    return false;
}

// The double-float update of the four cells of row gz, from the operator value S(U^n) (high part
// sh, low part slo, as lane pairs): U^{n+1} = 2U^n - U^{n-1} + [(a - 2)U^n + (b + 1)U^{n-1}] + kq S,
// the point source when it falls in these cells, and the stores of both planes of U^{n+1} and of
// the history (S times q.hist_scale, the operator with the textbook weights, rounded once).
template <int MODE>
__device__ __forceinline__ void comp_finish_row(const StepParams &p, const CompParams &q, const MapGrid &mg,
                                                bool interior, const int (&xd)[4], int gx, int gz,
                                                long long shot_off, float4 uh4, float4 ul4, float4 ph4, float4 pl4,
                                                float4 kh4, float4 kl4, const float2 (&sh)[2],
                                                const float2 (&slo)[2], int src_z, int src_x, float src_hi,
                                                float src_lo)
{
    float2 nh[2], nl[2], lap[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 uh = lane2(uh4, h), ul = lane2(ul4, h), pvh = lane2(ph4, h), pvl = lane2(pl4, h);
        const float2 kqh = lane2(kh4, h), kql = lane2(kl4, h);
        // 2 U^n - U^{n-1}
        float2 th, te;
        two_sum2(__fmul2_rn(make_float2(2.f, 2.f), uh), neg2(pvh), th, te);
        float2 tl = __fadd2_rn(te, __ffma2_rn(make_float2(2.f, 2.f), ul, neg2(pvl)));
        // + kq S(U)
        float2 qh, qe;
        two_prod2(kqh, sh[h], qh, qe);
        const float2 ql = __ffma2_rn(kqh, slo[h], __ffma2_rn(kql, sh[h], qe));
        float2 n1, ne;
        two_sum2(th, qh, n1, ne);
        float2 n2 = __fadd2_rn(__fadd2_rn(ne, tl), ql);
        if (!interior) {   // + (a - 2) U^n + (b + 1) U^{n-1}, coefficients hi + lo per depth pair
            const float4 *trow = q.damp + layer_depth(gz, p.P, mg.Nz) * (p.P + 1);
            const float4 c0 = __ldg(trow + xd[2 * h]), c1 = __ldg(trow + xd[2 * h + 1]);
            const float2 ah = make_float2(c0.x, c1.x), al = make_float2(c0.y, c1.y);
            const float2 bh2 = make_float2(c0.z, c1.z), bl2 = make_float2(c0.w, c1.w);
            float2 p1, e1, p2, e2, dh, de;
            two_prod2(ah, uh, p1, e1);
            two_prod2(bh2, pvh, p2, e2);
            two_sum2(p1, p2, dh, de);
            float2 dl = __fadd2_rn(de, __fadd2_rn(e1, e2));
            dl = __ffma2_rn(ah, ul, __ffma2_rn(al, uh, __ffma2_rn(bh2, pvl, __ffma2_rn(bl2, pvh, dl))));
            float2 m1, me;
            two_sum2(n1, dh, m1, me);
            n1 = m1;
            n2 = __fadd2_rn(n2, __fadd2_rn(me, dl));
        }
        two_sum2(n1, n2, nh[h], nl[h]);   // renormalise
        // Lap(U^n) with the textbook weights for the imaging condition, rounded once
        lap[h] = __ffma2_rn(sh[h], make_float2(q.hist_scale, q.hist_scale),
                            __fmul2_rn(slo[h], make_float2(q.hist_scale, q.hist_scale)));
    }
    float4 vh = f4(nh[0], nh[1]), vl = f4(nl[0], nl[1]), lv = f4(lap[0], lap[1]);
    // point source of step n at the transmit node (one cell of one thread)
    if (src_z == gz && src_x >= gx && src_x < gx + 4) {
        auto add_src = [&](float &h, float &l) {
            float a, b;
            two_sum(h, src_hi, a, b);
            const float lo = __fadd_rn(l, __fadd_rn(b, src_lo));
            two_sum(a, lo, h, l);
        };
        if (src_x == gx) add_src(vh.x, vl.x);
        else if (src_x == gx + 1) add_src(vh.y, vl.y);
        else if (src_x == gx + 2) add_src(vh.z, vl.z);
        else add_src(vh.w, vl.w);
    }
    if (gx >= mg.nxp || gz >= mg.nzp) return;
    if (gx + 4 > mg.nxp) {   // lanes past the last column stay zero (outside the map's grid)
        if (gx + 1 >= mg.nxp) { vh.y = 0.f; vl.y = 0.f; lv.y = 0.f; }
        if (gx + 2 >= mg.nxp) { vh.z = 0.f; vl.z = 0.f; lv.z = 0.f; }
        vh.w = 0.f; vl.w = 0.f; lv.w = 0.f;
    }
    const long long o = shot_off + static_cast<long long>(gz) * p.pitch + gx;
    st4(p.out + o, vh);
    st4(q.out_lo + o, vl);
    if (MODE == kFwdSampleHist || MODE == kFwdHist) st4_stream(p.hist + o, lv);
}

// Receivers of this tile: (hi, lo) of U^n from the boxes (row stride sx, halo hx).
template <int MODE>
__device__ __forceinline__ void comp_sample(const StepParams &p, const CompParams &q, int s, int tx_idx, int x0,
                                            int z0, const float *bh, const float *bl, int sx, int hx)
{
    if (MODE == kFwdSample || MODE == kFwdSampleHist) {
        const int2 rx_range = __ldg(p.rx_tab + tx_idx * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x);
        const int cnt = (rx_range.x >= 0 && rx_range.y >= 0 && rx_range.x + rx_range.y <= p.n_rx) ? rx_range.y : 0;
        for (int e = static_cast<int>(threadIdx.x); e < cnt; e += static_cast<int>(blockDim.x)) {
            const int r = __ldg(p.rx_sorted + tx_idx * p.n_rx + rx_range.x + e);
            const int node = (r >= 0 && r < p.n_rx) ? __ldg(p.smp_node + tx_idx * p.n_rx + r) : -1;
            const int zn = node >> 16, xn = node & 0xffff;
            if (node < 0 || zn < z0 || zn >= z0 + kCompTileZ || xn < x0 || xn >= x0 + kTileX) {
                raise_status(p.status, DUFWI_ERR_GEOMETRY);
                continue;
            }
            const long long co = (static_cast<long long>(s) * p.nt + p.step) * p.n_rx + r;
            const int bo = (zn - z0 + hx) * sx + (xn - x0 + hx);
            p.cd[co] = bh[bo];
            if (q.cd_lo) q.cd_lo[co] = bl[bo];
        }
    }
}

template <int R, int MODE>
__global__ void __launch_bounds__(128, 3) comp_step_kernel(const __grid_constant__ CompMaps tm, const StepParams p,
                                                           const CompParams q)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;

    const int tid = threadIdx.x;
    const int s = p.shot0 + blockIdx.z;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * kCompTileZ;
    const int tx_idx = s % p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *bh = smem;                      // U_hi^n box
    float *bl = bh + kCompBox;             // U_lo^n box
    float *ph = bl + kCompBox;             // U_hi^{n-1}
    float *pl = ph + kCompTile;            // U_lo^{n-1}
    float *kh = pl + kCompTile;            // kq_hi
    float *kl = kh + kCompTile;            // kq_lo
    const MapGrid mg = map_grid(p, s / p.n_tx);
    if (x0 >= mg.nxp || z0 >= mg.nzp) return;

    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, kCompBytes);
    }
    __syncthreads();   // the barrier is initialised before any thread polls it
    grid_dependency_wait();
    if (tid == 0) {
        tma_load_3d(bh, &tm.hi_box, &bar, x0 - kHalo, z0 - kHalo, s);
        tma_load_3d(bl, &tm.lo_box, &bar, x0 - kHalo, z0 - kHalo, s);
        tma_load_3d(ph, &tm.hi_tile, &bar, x0, z0, s);
        tma_load_3d(pl, &tm.lo_tile, &bar, x0, z0, s);
        tma_load_3d(kh, &tm.kq_hi, &bar, x0, z0, s / p.n_tx);
        tma_load_3d(kl, &tm.kq_lo, &bar, x0, z0, s / p.n_tx);
    }
    grid_dependents_launch();

    const int lx = (tid & 15) * 4;
    const int lz = (tid >> 4) * 4;
    const int gx = x0 + lx;
    const bool interior = region_interior(p, mg, x0, z0, kTileX, kCompTileZ);
    int xd[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, mg.Nx);
    // the transmit node of this shot (a point source; at most one per shot)
    const int src_node = __ldg(p.inj_node + tx_idx);
    const int src_z = src_node >> 16, src_x = src_node & 0xffff;
    // the source sample w[n] dt^2/dx^2 as hi + lo (dt^2/dx^2 itself as inj_scale + src_lo)
    const float w = __ldg(p.inj_val + static_cast<long long>(p.wav_per_tx ? tx_idx : 0) * p.nt + p.step);
    const float src_hi = __fmul_rn(w, p.inj_scale);
    const float src_lo = __fmaf_rn(w, q.src_lo, __fmaf_rn(w, p.inj_scale, -src_hi));

    if (!comp_wait(&bar, p)) return;

#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        const int rz = lz + j;          // row within the tile
        const int gz = z0 + rz;
        float2 sh[2], se[2], sl[2], dummy[2];
        stencil_row<R, true>(bh, kHalo + lx, kHalo + rz, sh, se);
        stencil_row<R, false>(bl, kHalo + lx, kHalo + rz, sl, dummy);
        const float4 uh4 = ld4s(bh + (kHalo + rz) * kBoxX + kHalo + lx);
        const float4 ul4 = ld4s(bl + (kHalo + rz) * kBoxX + kHalo + lx);
        const int to = rz * kTileX + lx;
        float2 slo[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) slo[h] = __fadd2_rn(se[h], sl[h]);   // low part of S(U)
        comp_finish_row<MODE>(p, q, mg, interior, xd, gx, gz, shot_off, uh4, ul4, ld4s(ph + to), ld4s(pl + to),
                              ld4s(kh + to), ld4s(kl + to), sh, slo, src_z, src_x, src_hi, src_lo);
    }

    comp_sample<MODE>(p, q, s, tx_idx, x0, z0, bh, bl, kBoxX, kHalo);
}

// ---- compensated variable-density step ------------------------------------------------------
// The staggered operator of Eq. 1, G = D-_x(b_x D+_x u) + D-_z(b_z D+_z u), in the same double-float
// arithmetic: integer staggered weights s'_k = S s_k (S = 1, 24, 1920, 107520 for orders 2 to 8:
// 1; 27, -1; 2250, -125, 9; 128625, -8575, 1029, -75), so the operator is scaled by S^2, which
// kq = kappa' / S^2 absorbs (kappa' = rho C^2 dt^2 / (dx^2 (1 + D dt))). The buoyancies b are FP64
// values split into hi + lo. A flux b D+u is formed with TwoSum / TwoProd on U_hi (the error terms
// summed in FP32), D+u_lo in plain FP32, and a double-float product with b; the divergence takes
// double-float differences of fluxes, TwoProd by the integer weights and TwoSum accumulation.
//
// Tile scheme: 64 x 32 output tiles, 128 threads, a 4 x 4 block per thread (the variable-density
// kernel's): the 80 x 48 boxes of U_hi^n and U_lo^n (halo 8), the 72 x 32 x-buoyancy and 64 x 40
// z-buoyancy tiles as hi and lo planes, and the 64 x 32 tiles of U^{n-1} and kq (hi, lo).
constexpr int kCvBox = kVBoxX * kVBoxZ;   // 80 x 48
constexpr int kCvFx = kVFxX * kVTileZ;    // 72 x 32
constexpr int kCvFz = kTileX * kVFzZ;     // 64 x 40
constexpr uint32_t kCvBytes = (2 * kCvBox + 2 * kCvFx + 2 * kCvFz + 4 * kCompTile) * sizeof(float);

template <int R>
__device__ __forceinline__ float stag_int_weight(int k)
{
    if (R == 1) return 1.0f;
    if (R == 2) return k == 1 ? 27.0f : -1.0f;
    if (R == 3) return k == 1 ? 2250.0f : (k == 2 ? -125.0f : 9.0f);
    return k == 1 ? 128625.0f : (k == 2 ? -8575.0f : (k == 3 ? 1029.0f : -75.0f));
}

struct DF {   // double-float value hi + lo
    float h, l;
};

// b D+u at a half point: u_hi values a[k - 1] (upper) and c[k - 1] (lower) of the R differences
// u[+k] - u[-k + 1], their low parts al, cl; b as (bh, bl).
template <int R>
__device__ __forceinline__ DF comp_flux(const float (&a)[R], const float (&c)[R], const float (&al)[R],
                                        const float (&cl)[R], float bh, float bl)
{
    float acc = 0.f, err = 0.f, lo = 0.f;
#pragma unroll
    for (int k = 1; k <= R; ++k) {
        const float w = stag_int_weight<R>(k);
        float d, e1, pr, e2;
        two_sum(a[k - 1], -c[k - 1], d, e1);
        pr = __fmul_rn(w, d);
        e2 = __fmaf_rn(w, d, -pr);
        if (k == 1) {
            acc = pr;
            err = __fmaf_rn(w, e1, e2);
        } else {
            float s2, e3;
            two_sum(acc, pr, s2, e3);
            acc = s2;
            err = __fmaf_rn(w, e1, __fadd_rn(err, __fadd_rn(e2, e3)));
        }
        lo = __fmaf_rn(w, __fsub_rn(al[k - 1], cl[k - 1]), lo);
    }
    const float dl = __fadd_rn(err, lo);
    DF f;
    f.h = __fmul_rn(bh, acc);
    f.l = __fmaf_rn(bh, dl, __fmaf_rn(bl, acc, __fmaf_rn(bh, acc, -f.h)));
    return f;
}

// acc += w (x - y) for double-float x, y and an integer weight w (error-free up to the low terms)
__device__ __forceinline__ void comp_div_tap(DF &acc, float w, DF x, DF y, bool first)
{
    float s, e;
    two_sum(x.h, -y.h, s, e);
    const float slo = __fadd_rn(e, __fsub_rn(x.l, y.l));
    const float p = __fmul_rn(w, s);
    const float plo = __fmaf_rn(w, slo, __fmaf_rn(w, s, -p));
    if (first) {
        acc.h = p;
        acc.l = plo;
    } else {
        float s2, e2;
        two_sum(acc.h, p, s2, e2);
        acc.h = s2;
        acc.l = __fadd_rn(acc.l, __fadd_rn(e2, plo));
    }
}

template <int R, int MODE>
__global__ void __launch_bounds__(128, 2) comp_vd_step_kernel(const __grid_constant__ CompVdMaps tm, const StepParams p,
                                                              const CompParams q)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ alignas(8) uint64_t bar;

    const int tid = threadIdx.x;
    const int s = p.shot0 + blockIdx.z;
    const int x0 = blockIdx.x * kTileX;
    const int z0 = blockIdx.y * kVTileZ;
    const int tx_idx = s % p.n_tx;
    const int map = s / p.n_tx;
    const long long shot_off = static_cast<long long>(s) * p.slice;
    float *bh = smem;                      // U_hi^n box (80 x 48)
    float *bl = bh + kCvBox;               // U_lo^n box
    float *xh = bl + kCvBox;               // x-buoyancies hi (72 x 32)
    float *xl = xh + kCvFx;
    float *zh = xl + kCvFx;                // z-buoyancies hi (64 x 40)
    float *zl = zh + kCvFz;
    float *ph = zl + kCvFz;                // U_hi^{n-1}
    float *pl = ph + kCompTile;
    float *kh = pl + kCompTile;            // kq hi, lo
    float *kl = kh + kCompTile;
    const MapGrid mg = map_grid(p, map);
    if (x0 >= mg.nxp || z0 >= mg.nzp) return;

    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, kCvBytes);
    }
    __syncthreads();
    grid_dependency_wait();
    if (tid == 0) {
        tma_load_3d(bh, &tm.hi_box, &bar, x0 - kVHalo, z0 - kVHalo, s);
        tma_load_3d(bl, &tm.lo_box, &bar, x0 - kVHalo, z0 - kVHalo, s);
        tma_load_3d(xh, &tm.bx_hi, &bar, x0 - kHalo, z0, map);
        tma_load_3d(xl, &tm.bx_lo, &bar, x0 - kHalo, z0, map);
        tma_load_3d(zh, &tm.bz_hi, &bar, x0, z0 - kHalo, map);
        tma_load_3d(zl, &tm.bz_lo, &bar, x0, z0 - kHalo, map);
        tma_load_3d(ph, &tm.hi_tile, &bar, x0, z0, s);
        tma_load_3d(pl, &tm.lo_tile, &bar, x0, z0, s);
        tma_load_3d(kh, &tm.kq_hi, &bar, x0, z0, map);
        tma_load_3d(kl, &tm.kq_lo, &bar, x0, z0, map);
    }
    grid_dependents_launch();

    const int lx = (tid & 15) * 4;
    const int lz = (tid >> 4) * 4;
    const int gx = x0 + lx;
    const bool interior = region_interior(p, mg, x0, z0, kTileX, kVTileZ);
    int xd[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xd[i] = layer_depth(gx + i, p.P, mg.Nx);
    const int src_node = __ldg(p.inj_node + tx_idx);
    const int src_z = src_node >> 16, src_x = src_node & 0xffff;
    const float w = __ldg(p.inj_val + static_cast<long long>(p.wav_per_tx ? tx_idx : 0) * p.nt + p.step);
    const float src_hi = __fmul_rn(w, p.inj_scale);
    const float src_lo = __fmaf_rn(w, q.src_lo, __fmaf_rn(w, p.inj_scale, -src_hi));

    if (!comp_wait(&bar, p)) return;

    // z-direction first: flux rows f = 0..10 (half points z0 - 4 + lz + f + 1/2, z-buoyancy rows
    // lz + f) of the four columns; box rows lz + f + 4 + k and lz + f + 5 - k; output row j takes
    // +w_k from flux row j + k + 3 and -w_k from flux row j - k + 4.
    DF gz_acc[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        DF fz[11];
#pragma unroll
        for (int f = 0; f < 11; ++f) {
            float a[R], cc[R], al[R], cl[R];
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                const int up = (lz + f + 4 + k) * kVBoxX + lx + kVHalo + c;
                const int dn = (lz + f + 5 - k) * kVBoxX + lx + kVHalo + c;
                a[k - 1] = bh[up];
                cc[k - 1] = bh[dn];
                al[k - 1] = bl[up];
                cl[k - 1] = bl[dn];
            }
            const int bo = (lz + f) * kTileX + lx + c;
            fz[f] = comp_flux<R>(a, cc, al, cl, zh[bo], zl[bo]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int k = 1; k <= R; ++k)
                comp_div_tap(gz_acc[j][c], stag_int_weight<R>(k), fz[j + k + 3], fz[j - k + 4], k == 1);
        }
    }

#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        const int rz = lz + j;
        const int gz = z0 + rz;
        const int brow = (rz + kVHalo) * kVBoxX + lx;   // box row of this output row, column lx - 8 + 8
        // x-direction: fluxes h = 0..10 at half points x0 - 4 + lx + h + 1/2 (x-buoyancy columns
        // lx + h), from box columns lx + h + 4 + k and lx + h + 5 - k
        DF fx[11];
#pragma unroll
        for (int h = 0; h < 11; ++h) {
            float a[R], cc[R], al[R], cl[R];
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                a[k - 1] = bh[brow + h + 4 + k];
                cc[k - 1] = bh[brow + h + 5 - k];
                al[k - 1] = bl[brow + h + 4 + k];
                cl[k - 1] = bl[brow + h + 5 - k];
            }
            const int bo = rz * kVFxX + lx + h;
            fx[h] = comp_flux<R>(a, cc, al, cl, xh[bo], xl[bo]);
        }
        float2 sh[2], slo[2];
        float gh[4], gl[4];
#pragma unroll
        for (int qx = 0; qx < 4; ++qx) {
            DF gx_acc;
#pragma unroll
            for (int k = 1; k <= R; ++k)
                comp_div_tap(gx_acc, stag_int_weight<R>(k), fx[qx + k + 3], fx[qx - k + 4], k == 1);
            // G = Gx + Gz
            float s2, e2;
            two_sum(gx_acc.h, gz_acc[j][qx].h, s2, e2);
            gh[qx] = s2;
            gl[qx] = __fadd_rn(e2, __fadd_rn(gx_acc.l, gz_acc[j][qx].l));
        }
        sh[0] = make_float2(gh[0], gh[1]);
        sh[1] = make_float2(gh[2], gh[3]);
        slo[0] = make_float2(gl[0], gl[1]);
        slo[1] = make_float2(gl[2], gl[3]);
        const int to = rz * kTileX + lx;
        comp_finish_row<MODE>(p, q, mg, interior, xd, gx, gz, shot_off, ld4s(bh + brow + kVHalo),
                              ld4s(bl + brow + kVHalo), ld4s(ph + to), ld4s(pl + to), ld4s(kh + to), ld4s(kl + to),
                              sh, slo, src_z, src_x, src_hi, src_lo);
    }

    comp_sample<MODE>(p, q, s, tx_idx, x0, z0, bh, bl, kVBoxX, kVHalo);
}

// Buoyancies of the compensated variable-density step as hi + lo: b = 2 / (rho + rho') at the x and
// z half points in FP64 (as setup_kappa_kernel forms them, whose FP32 rounding is the hi part), and
// kq = rho C^2 (dt/dx)^2 / ((1 + D dt) S^2) with density and SoS edge-replicated into the layer.
__global__ void setup_comp_vd_kernel(const float *sos, const float *density, float *kq_hi, float *kq_lo, float *bxl,
                                     float *bzl, int NxE, int NzE, int P, int nzpE, int pitch, double r2_over_s2,
                                     double d0, double dt, const int2 *map_dims)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int b = blockIdx.z;
    if (x >= pitch) return;
    const int Nx = map_dims ? map_dims[b].x : NxE, Nz = map_dims ? map_dims[b].y : NzE;
    const int nxp = Nx + 2 * P, nzp = Nz + 2 * P;
    const long long o = (static_cast<long long>(b) * nzpE + z) * pitch + x;
    if (x >= nxp || z >= nzp) {
        kq_hi[o] = 0.f;
        kq_lo[o] = 0.f;
        bxl[o] = 0.f;
        bzl[o] = 0.f;
        return;
    }
    auto src_of = [&](int xx, int zz) {
        const int xs = min(max(xx - P, 0), Nx - 1), zs = min(max(zz - P, 0), Nz - 1);
        return (static_cast<long long>(b) * NzE + zs) * NxE + xs;
    };
    const long long src = src_of(x, z);
    const double C = sos[src];
    const double rho = density[src];
    const double rx = x + 1 < nxp ? static_cast<double>(density[src_of(x + 1, z)]) : rho;
    const double rz = z + 1 < nzp ? static_cast<double>(density[src_of(x, z + 1)]) : rho;
    const double bx = x + 1 < nxp ? 2.0 / (rho + rx) : 0.0;
    const double bz = z + 1 < nzp ? 2.0 / (rho + rz) : 0.0;
    bxl[o] = static_cast<float>(bx - static_cast<double>(static_cast<float>(bx)));
    bzl[o] = static_cast<float>(bz - static_cast<double>(static_cast<float>(bz)));
    const int dxl = x < P ? P - x : (x > P + Nx - 1 ? x - (P + Nx - 1) : 0);
    const int dzl = z < P ? P - z : (z > P + Nz - 1 ? z - (P + Nz - 1) : 0);
    const double xx = static_cast<double>(dxl) / P, zz = static_cast<double>(dzl) / P;
    const double D = d0 * xx * xx + d0 * zz * zz;
    const double v = rho * C * C * r2_over_s2 / (1.0 + D * dt);
    const float hi = static_cast<float>(v);
    kq_hi[o] = hi;
    kq_lo[o] = static_cast<float>(v - static_cast<double>(hi));
}

template <int R, int MODE>
cudaError_t launch_comp_vd_rm(const CompVdMaps &tm, const StepParams &p, const CompParams &q, cudaStream_t st)
{
    static DeviceCache dc;
    cudaError_t e = configure_kernel(comp_vd_step_kernel<R, MODE>, kCvBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + kVTileZ - 1) / kVTileZ, p.n_shots);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = kCvBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, comp_vd_step_kernel<R, MODE>, tm, p, q);
}

template <int R>
cudaError_t launch_comp_vd_r(int mode, const CompVdMaps &tm, const StepParams &p, const CompParams &q,
                             cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_comp_vd_rm<R, kFwdSample>(tm, p, q, st);
    case kFwdSampleHist: return launch_comp_vd_rm<R, kFwdSampleHist>(tm, p, q, st);
    case kFwdHist: return launch_comp_vd_rm<R, kFwdHist>(tm, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

// kq = kappa' / s_R = C^2 (dt/dx)^2 / ((1 + D dt) s_R) on the padded grid, in FP64, split into
// hi + lo (C edge-replicated into the absorbing layer, as for kappa').
__global__ void setup_kq_kernel(const float *sos, float *kq_hi, float *kq_lo, int NxE, int NzE, int P, int nzpE,
                                int pitch, double r2_over_s, double d0, double dt, const int2 *map_dims)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int b = blockIdx.z;
    if (x >= pitch) return;
    const int Nx = map_dims ? map_dims[b].x : NxE, Nz = map_dims ? map_dims[b].y : NzE;
    const int nxp = Nx + 2 * P, nzp = Nz + 2 * P;
    const long long o = (static_cast<long long>(b) * nzpE + z) * pitch + x;
    if (x >= nxp || z >= nzp) {
        kq_hi[o] = 0.f;
        kq_lo[o] = 0.f;
        return;
    }
    const int xs = min(max(x - P, 0), Nx - 1), zs = min(max(z - P, 0), Nz - 1);
    const double C = sos[(static_cast<long long>(b) * NzE + zs) * NxE + xs];
    const int dxl = x < P ? P - x : (x > P + Nx - 1 ? x - (P + Nx - 1) : 0);
    const int dzl = z < P ? P - z : (z > P + Nz - 1 ? z - (P + Nz - 1) : 0);
    const double xx = static_cast<double>(dxl) / P, zz = static_cast<double>(dzl) / P;
    const double D = d0 * xx * xx + d0 * zz * zz;
    const double v = C * C * r2_over_s / (1.0 + D * dt);
    const float hi = static_cast<float>(v);
    kq_hi[o] = hi;
    kq_lo[o] = static_cast<float>(v - static_cast<double>(hi));
}

template <int R, int MODE>
cudaError_t launch_comp_rm(const CompMaps &tm, const StepParams &p, const CompParams &q, cudaStream_t st)
{
    static DeviceCache dc;
    cudaError_t e = configure_kernel(comp_step_kernel<R, MODE>, kCompBytes, dc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nxp + kTileX - 1) / kTileX, (p.nzp + kCompTileZ - 1) / kCompTileZ, p.n_shots);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = kCompBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, comp_step_kernel<R, MODE>, tm, p, q);
}

template <int R>
cudaError_t launch_comp_r(int mode, const CompMaps &tm, const StepParams &p, const CompParams &q, cudaStream_t st)
{
    switch (mode) {
    case kFwdSample: return launch_comp_rm<R, kFwdSample>(tm, p, q, st);
    case kFwdSampleHist: return launch_comp_rm<R, kFwdSampleHist>(tm, p, q, st);
    case kFwdHist: return launch_comp_rm<R, kFwdHist>(tm, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

double comp_weight_scale(int order)
{
    switch (order) {
    case 2: return 1.0;
    case 4: return 12.0;
    case 6: return 180.0;
    case 8: return 5040.0;
    default: return 0.0;
    }
}

cudaError_t launch_comp_step(int radius, int mode, const CompMaps &tm, const StepParams &p, const CompParams &q,
                             cudaStream_t st)
{
    if (p.tile_z != kCompTileZ) return cudaErrorInvalidValue;
    switch (radius) {
    case 1: return launch_comp_r<1>(mode, tm, p, q, st);
    case 2: return launch_comp_r<2>(mode, tm, p, q, st);
    case 3: return launch_comp_r<3>(mode, tm, p, q, st);
    case 4: return launch_comp_r<4>(mode, tm, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

double comp_stagger_scale(int order)
{
    switch (order) {
    case 2: return 1.0;
    case 4: return 24.0;
    case 6: return 1920.0;
    case 8: return 107520.0;
    default: return 0.0;
    }
}

cudaError_t launch_comp_vd_step(int radius, int mode, const CompVdMaps &tm, const StepParams &p, const CompParams &q,
                                cudaStream_t st)
{
    if (p.tile_z != kVTileZ) return cudaErrorInvalidValue;
    switch (radius) {
    case 1: return launch_comp_vd_r<1>(mode, tm, p, q, st);
    case 2: return launch_comp_vd_r<2>(mode, tm, p, q, st);
    case 3: return launch_comp_vd_r<3>(mode, tm, p, q, st);
    case 4: return launch_comp_vd_r<4>(mode, tm, p, q, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_setup_comp_vd(const float *sos, const float *density, float *kq_hi, float *kq_lo, float *bx_lo,
                                 float *bz_lo, int n_maps, int Nx, int Nz, int P, int nzp, int pitch, double dt_over_dx,
                                 double stagger_scale, double d0, double dt, const int2 *map_dims, cudaStream_t st)
{
    dim3 grid((pitch + 127) / 128, nzp, n_maps);
    setup_comp_vd_kernel<<<grid, 128, 0, st>>>(sos, density, kq_hi, kq_lo, bx_lo, bz_lo, Nx, Nz, P, nzp, pitch,
                                               dt_over_dx * dt_over_dx / (stagger_scale * stagger_scale), d0, dt,
                                               map_dims);
    return cudaGetLastError();
}

cudaError_t launch_setup_kq(const float *sos, float *kq_hi, float *kq_lo, int n_maps, int Nx, int Nz, int P, int nzp,
                            int pitch, double dt_over_dx, double weight_scale, double d0, double dt,
                            const int2 *map_dims, cudaStream_t st)
{
    dim3 grid((pitch + 127) / 128, nzp, n_maps);
    setup_kq_kernel<<<grid, 128, 0, st>>>(sos, kq_hi, kq_lo, Nx, Nz, P, nzp, pitch,
                                          dt_over_dx * dt_over_dx / weight_scale, d0, dt, map_dims);
    return cudaGetLastError();
}

}  // namespace dufwi
