// dufwi_internal.h -- shared declarations of the sm_103a kernels and the host-side ABI code.
//
// Data layout in device memory (one workspace, carved by the host code):
//   field  [S][nzp][pitch] float, S = n_maps * n_tx shots; the padded grid is nzp x nxp with
//          nxp = nx + 2P and nzp = nz + 2P; pitch = nxp rounded up to 8 floats (32-byte rows).
//          Columns nxp..pitch-1 are never read by the stencil (the TMA box treats x >= nxp as
//          outside the tensor, i.e. zero).
//   kappa  [n_maps][nzp][pitch] float: kappa' = C^2 dt^2 / (dx^2 (1 + D dt)), the Eq. 2
//          coefficient with the 1/dx^2 of the Laplacian folded in. It is computed once per call
//          in FP64 and rounded once.
//   bx, bz [n_maps][nzp][pitch] float: buoyancy 1/rho at the half points (x + 1/2, z) and
//          (x, z + 1/2), 2 / (rho + rho_neighbour) in FP64 rounded once; 0 past the last node of
//          a row (bx) or column (bz). Used only with a density map (variable-density operator).
//   node   packed (zp << 16) | xp padded-grid node of an element.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dufwi.h"

#include <atomic>

namespace dufwi {

// Kernel attributes (dynamic shared memory, carveout) and resident-CTA counts belong to a device:
// launchers keep them per device index, so a process may drive several GPUs and several host
// threads may launch at once (a repeated attribute call is harmless; the cached values are the
// same whichever thread stores them).
constexpr int kMaxDevices = 64;

struct DeviceCache {
    std::atomic<uint64_t> configured{0};        // bit d: attributes set on device d
    std::atomic<int> resident[kMaxDevices] = {};  // co-resident CTAs on device d (0: not computed)
};

template <typename K>
inline cudaError_t configure_kernel(K kernel, uint32_t smem_bytes, DeviceCache &dc, int *device = nullptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (device) *device = dev;
    const uint64_t bit = 1ull << dev;
    if (dc.configured.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) dc.configured.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// CTAs of `kernel` (threads per CTA, dynamic shared memory) that fit on the current device at once.
template <typename K>
inline cudaError_t resident_ctas(K kernel, int threads, uint32_t smem_bytes, DeviceCache &dc, int *out)
{
    int dev = 0;
    cudaError_t e = configure_kernel(kernel, smem_bytes, dc, &dev);
    if (e != cudaSuccess) return e;
    int n = dc.resident[dev].load(std::memory_order_acquire);
    if (n == 0) {
        int sms = 0, per_sm = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem_bytes)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        n = per_sm * sms;
        dc.resident[dev].store(n, std::memory_order_release);
    }
    *out = n;
    return cudaSuccess;
}

constexpr int kTileX = 64;                    // output tile width (x, contiguous)
constexpr int kHalo = 4;                      // halo loaded on every side (max stencil radius)
constexpr int kBoxX = kTileX + 2 * kHalo;     // TMA box: 72 floats = 288 bytes per row
constexpr int kTileZDefault = 32;             // output tile height (z): 32 or 64

// Variable-density step (staggered operator of Eq. 1): 64 x 32 output tiles, a halo of 8 for the
// U^n box (two staggered differences of radius up to 4) and of 4 for the half-point buoyancies.
constexpr int kVHalo = 2 * kHalo;             // 8
constexpr int kVTileZ = 32;
constexpr int kVBoxX = kTileX + 2 * kVHalo;   // 80 floats = 320 bytes per row
constexpr int kVBoxZ = kVTileZ + 2 * kVHalo;  // 48
constexpr int kVFxX = kTileX + 2 * kHalo;     // 72 x-half-points per row: x0 - 4 + i + 1/2
constexpr int kVFzZ = kVTileZ + 2 * kHalo;    // 40 z-half-point rows: z0 - 4 + j + 1/2

// Step kernel variants.
enum StepMode : int {
    kFwdSample = 0,      // forward step, record receivers (simulation, first pass with snapshots)
    kFwdSampleHist = 1,  // forward step, record receivers, keep Lap(U^n) (store-all first pass)
    kFwdHist = 2,        // forward step, keep Lap(U^n) (recompute of one checkpoint segment)
    kAdjoint = 3,        // adjoint step with residual injection and zero-lag imaging
    kBorn = 4,           // linearised (Born) step: dU^{n+1} = Eq. 2 on dU + dkappa' Lap(U^n), receivers
};

// Second-order sweep kinds (so_step_kernel).
enum SoKind : int {
    kSoBorn = 0,         // Born step that also keeps Lap(dU^n); receivers sampled when cd is set
    kSoAdj = 1,          // adjoint step, two imaging sums (with Lap(U^{m-1}) and Lap(dU^{m-1})), keeps Lap(mu^{m+1})
    kSoBornAdj = 2,      // derivative of the adjoint step along v: source dkappa' Lap(mu^{m+1}), imaging with Lap(U^{m-1})
};

// Tensor maps of one step launch (all FP32, no swizzle, zero fill outside the tensor):
//   cur_box   field being read with halo: dims (nxp, nzp, S), box 72 x (TZ + 8) x 1
//   out_tile  field updated in place: dims (nxp, nzp, S), box 64 x TZ x 1
//   kap_tile  kappa': dims (nxp, nzp, n_maps), box 64 x TZ x 1
//   hist_tile history ring: dims (nxp, nzp, S, n_hist), box 64 x TZ x 1 x 1 (adjoint only)
//   grad_tile imaging sums: dims (nxp, nzp, S), box 64 x TZ x 1 (adjoint); in the Born step the
//             perturbation dkappa': dims (nxp, nzp, n_maps), box 64 x TZ x 1
//   bx_tile, bz_tile  variable-density step only: buoyancies, dims (nxp, nzp, n_maps), boxes
//             72 x 32 x 1 (from x0 - 4) and 64 x 40 x 1 (from z0 - 4); cur_box is then 80 x 48
struct StepMaps {
    CUtensorMap cur_box, out_tile, kap_tile, hist_tile, grad_tile, bx_tile, bz_tile;
};

// Convolutional PML (CPML) step: the staggered operator with one memory variable per first
// difference and axis. Forward: psi at half points (read over the 72 x 32 / 64 x 40 half-point
// tiles of the previous step's buffer, written for the tile's own half points into the other
// buffer), xi at nodes (own tile, in place). Adjoint: phi (adjoint of psi) like psi, chi (adjoint
// of xi) read over 80 x 32 / 64 x 48 node boxes (halo 8 along its axis) of the previous buffer
// and written for the own nodes into the other.
struct CpmlMaps {
    CUtensorMap mem_hx, mem_hz;   // psi / phi: x half points 72 x 32 (from x0 - 4), z 64 x 40 (from z0 - 4)
    CUtensorMap mem_nx, mem_nz;   // forward xi: 64 x 32 own nodes; adjoint chi: 80 x 32 / 64 x 48 boxes
};

struct CpmlParams {
    float *hx_out, *hz_out;       // memory variables at half points, written (own half points)
    float *nx_out, *nz_out;       // memory variables at nodes, written (own nodes)
    const float *cx;              // [4][nxp]: a, b at x nodes, then a, b at x half points
    const float *cz;              // [4][nzp]: the same along z
};

struct StepParams {
    float *out;              // in: U^{n-1} (mu^{m+2}); out: U^{n+1} (mu^m), in place
    const float *kap;        // [n_maps][nzp][pitch]
    float *hist;             // forward: Lap(U^n) for this step; adjoint: Lap(U^{m-1})
    float *grad;             // adjoint: [S][nzp][pitch] running sum of mu^m * Lap(U^{m-1})
    const int *inj_node;     // forward: [n_tx] transmit nodes; adjoint: [n_tx][n_rx] receivers
    const float *inj_val;    // forward: wavelet [1 or n_tx][nt]; adjoint: source [S][nt][n_rx]
    const int *smp_node;     // forward: receivers [n_tx][n_rx]
    const int2 *rx_tab;      // [n_tx][tiles]: (first, count) of the receivers inside each tile
    const int *rx_sorted;    // [n_tx][n_rx]: receiver indices grouped by tile (row-major tiles)
    const int2 *rxe_tab;     // two-step kernel: (first, count) of the receivers inside each tile
                             // grown by 4 cells on every side
    const int *rxe_sorted;   // [n_tx][n_rxe]: receiver indices grouped by grown tile
    int n_rxe;               // row length of rxe_sorted
    float *out2;             // two-step kernel: U^{n+2} (mu^{m-1}); out holds U^{n+1} (mu^m)
    float *hist2;            // two-step kernel: Lap(U^{n+1}) (forward history)
    int hist_slot2;          // two-step adjoint: slot of Lap(U^{m-2})
    float *cd;               // forward: channel data [S][nt][n_rx] (sampled at U^n)
    int *status;             // device status word
    long long slice;         // nzp * pitch
    int nxp, nzp, pitch;
    int n_maps, n_tx, n_rx;
    int hist_slot;           // adjoint: slot of Lap(U^{m-1}) in the history ring
    int tile_z;              // output tile height TZ (32 or 64)
    int step;                // n (forward: produces U^{n+1}) or m (adjoint: produces mu^m)
    int nt;
    int wav_per_tx;
    float inj_scale;         // forward: dt^2/dx^2
    int P, Nx, Nz;           // absorbing-layer thickness and physical grid
    const int2 *map_dims;    // sized calls: [n_maps] (Nx, Nz) of each map; null for a uniform call
    const float2 *damp_tab;  // [P + 1][P + 1]: (a - 2, b + 1) at layer depths (dz, dx) in cells
    float c[5];              // central stencil weights, c[0] the centre weight of one axis
    float sw[4];             // staggered first-difference weights s_1..s_R (variable density)
    int early;               // one-step kernel: U^{n-1}, kappa' (and the history) may be loaded before
                             // the wait for the previous launch: neither of the last two launches
                             // wrote them (set by the host from the third step of a range on)
    int tile_class;          // CPML split: 0 every tile; 1 only tiles whose region grown by 8 cells
                             // lies inside the physical grid (no memory variables); 2 only the others
    int shot0, n_shots;      // this launch covers shots shot0 .. shot0 + n_shots - 1 (grid.z = n_shots)
    int min_ctas;            // one-step kernel, 8th order, 64 x 32 tiles: register-cap variant (0, 4 or 6)
};

// Compensated forward step (comp_step_kernel, 64 x 32 tiles): the field as hi + lo planes of FP32.
//   hi_box, lo_box    U^n planes read with halo: dims (nxp, nzp, S), box 72 x 40 x 1
//   hi_tile, lo_tile  U^{n-1} planes, updated in place to U^{n+1}: box 64 x 32 x 1
//   kq_hi, kq_lo      kappa' / s_R as hi + lo: dims (nxp, nzp, n_maps), box 64 x 32 x 1
struct CompMaps {
    CUtensorMap hi_box, lo_box, hi_tile, lo_tile, kq_hi, kq_lo;
};

// Compensated variable-density step (comp_vd_step_kernel, 64 x 32 tiles): the U^n planes read
// with halo 8 (boxes 80 x 48), U^{n-1} and kq tiles (64 x 32), the buoyancies as hi and lo planes
// (x: 72 x 32 from x0 - 4; z: 64 x 40 from z0 - 4; dims (nxp, nzp, n_maps)).
struct CompVdMaps {
    CUtensorMap hi_box, lo_box, hi_tile, lo_tile, kq_hi, kq_lo, bx_hi, bx_lo, bz_hi, bz_lo;
};

struct CompParams {
    float *out_lo;           // low plane of U^{n-1} in, of U^{n+1} out (StepParams::out is the high plane)
    float *cd_lo;            // low parts of the channel data [S][nt][n_rx], or null
    const float4 *damp;      // [P + 1][P + 1]: (a - 2) hi, lo, (b + 1) hi, lo at layer depths (dz, dx)
    float src_lo;            // low part of dt^2/dx^2 (StepParams::inj_scale is the high part)
    float hist_scale;        // 1 / s_R: the history holds Lap(U^n) with the textbook weights
};

// Second-order products (the derivative of the vector-Jacobian product along an SoS direction):
// tensor maps and extra arguments of so_step_kernel (64 x 32 tiles).
struct SoMaps {
    CUtensorMap cur_box, out_tile, kap_tile;   // the advanced field (box with halo, previous tile), kappa'
    CUtensorMap bx, bz;                        // variable density: half-point buoyancies (72 x 32, 64 x 40)
    CUtensorMap h1, h2;                        // histories [slot][S]: Lap(U^n), Lap(dU^n)
    CUtensorMap src;                           // Lap(mu^{m+1}) of the current adjoint step [S]
    CUtensorMap dk;                            // dkappa' [n_maps]
    CUtensorMap g1, g2;                        // running imaging sums [S]
};

struct SoParams {
    float *lap_out;          // Born: Lap(dU^n) (second-history slot); adjoint: Lap(mu^{m+1})
    float *sum1;             // adjoint: sum of mu^m Lap(U^{m-1}); Born-adjoint: sum of dmu^m Lap(U^{m-1})
    float *sum2;             // adjoint: sum of mu^m Lap(dU^{m-1})
    int h1_slot;             // slot of Lap(U^n) (Born) or Lap(U^{m-1}) (adjoint kinds) in h1
    int h2_slot;             // adjoint: slot of Lap(dU^{m-1}) in h2
    const float *dkap;       // CPML Born-adjoint (layer tiles): dkappa' [n_maps][nzp][pitch]
};

// Persistent sweep: n_steps consecutive steps of one sweep in a single cooperative launch. Work
// items are (local step i, tile k) in the order g = i * tiles + k; CTA b takes g = b, b + G, ...
// Before item (i, k) a CTA waits until tile k and its four neighbours in the same shot have
// completed i local steps (per-tile counters in flags, published with release semantics after
// the tile's stores); the smallest unfinished item therefore never waits, so all-resident CTAs
// cannot deadlock. The two field buffers alternate: local step i reads the current field through
// box[i & 1] and the previous one through tile[i & 1], and writes the new field in place of the
// previous one at out[i & 1].
struct SweepMaps {
    CUtensorMap box[2], tile[2], kap, hist, grad;
};

struct SweepParams {
    int n_steps;             // steps in this launch
    int step0;               // first step: forward n = step0 + i, adjoint m = step0 - i
    int tiles_x, tiles_z;    // tiles of one shot (64 x 32)
    int tiles;               // tiles of all shots
    int *flags;              // [tiles] local steps completed (zeroed before the launch)
    int *abort;              // set by a CTA whose wait ran out; every waiter then returns
    float *out[2];           // field written by local step i: out[i & 1]
    float *hist0;            // forward history: slot of step0 (stride hist_stride floats per step)
    long long hist_stride;
    int hist_slot0;          // adjoint: history slot of m - 1 for m = step0
    int stall_tile;          // test hook: this tile's wait can never be met (-1: none)
};

// Cluster-resident sweep (cluster_sweep_kernel): a range of steps of the compact stencil for
// grids small enough that one shot's fields fit in the shared memory of a cluster of kClusterCtas
// CTAs. CTA rank k of the cluster owns the padded rows [k H, (k + 1) H) of its shot; each step
// copies the 4 halo rows above and below from its neighbours' shared memory (distributed shared
// memory) and synchronises the cluster once. cur / prv: U^{n0}, U^{n0-1} (mu^{m0+1}, mu^{m0+2})
// read at the start; out_cur / out_prv receive the last two fields at the end.
constexpr int kClusterCtas = 8;
struct ClusterParams {
    const float *cur, *prv;
    float *out_cur, *out_prv;
    int n_steps;             // steps in this launch
    int step0;               // first step: forward n = step0 + i, adjoint m = step0 - i
    int H;                   // rows per CTA (a multiple of 4)
    int lpitch;              // shared-memory row stride (floats): 4 zero columns, nxp rounded to 4, 4 zero columns
    float *hist0;            // forward with history: Lap(U^{step0}); adjoint: Lap(U^{step0 - 1})
    long long hist_stride;   // floats between consecutive steps' history slots
};
// Shared memory of the cluster form per CTA (bytes) for a padded grid, or 0 when it does not fit.
size_t cluster_smem_bytes(int nxp, int nzp, int *H, int *lpitch);

// Host launchers (dufwi_kernels.cu). All return cudaGetLastError() of the launch.
cudaError_t launch_step(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st);
// Cluster-resident sweep of p.n_shots shots (modes kFwdSample, kFwdSampleHist, kFwdHist, kAdjoint).
cudaError_t launch_cluster_sweep(int radius, int mode, const StepParams &p, const ClusterParams &cp, cudaStream_t st);
// Multi-tile form of the one-step kernel (64 x 32 tiles, a grid of co-resident CTAs walking all
// tiles with two-stage TMA loads); same modes and results as launch_step with tile height 32.
cudaError_t launch_step_mt(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st);
// Two time steps per launch (core tiles 64 x 32; see step2_kernel).
cudaError_t launch_step2(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st);
constexpr int kPairTileZ = 32;   // core tile height of the two-step kernel (64 x 32 tiles)
// Persistent sweep (modes kFwdSample, kFwdSampleHist, kFwdHist, kAdjoint; 64 x 32 tiles). grid_ctas
// receives the grid used (all CTAs co-resident, cooperative launch).
cudaError_t launch_sweep(int radius, int mode, const SweepMaps &tm, const StepParams &p, const SweepParams &sp,
                         int *grid_ctas, cudaStream_t st);
// CPML step (modes kFwdSample, kFwdSampleHist, kFwdHist, kAdjoint; 64 x 32 tiles; the fields use
// the variable-density maps of StepMaps with cur_box 80 x 48).
cudaError_t launch_step_cpml(int radius, int mode, const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                             const CpmlParams &cp, cudaStream_t st);
// Variable-density step (modes kFwdSample, kFwdSampleHist, kFwdHist, kAdjoint, kBorn; 64 x 32 tiles).
cudaError_t launch_step_vd(int radius, int mode, const StepMaps &tm, const StepParams &p, cudaStream_t st);
// One step of the second-order sweeps (kinds kSoBorn, kSoAdj, kSoBornAdj; 64 x 32 tiles).
// vd: the staggered variable-density operator (cur_box 80 x 48 with halo 8, buoyancy maps set)
// instead of the compact Laplacian (cur_box 72 x 40).
// Second-order kinds on the CPML layer tiles (p.tile_class 2; the other tiles run launch_so_step
// with the staggered operator and p.tile_class 1). tm: cur_box (80 x 48 box of the advanced
// field), out_tile, kap_tile, bx_tile, bz_tile; hist_tile = the first history (4-D); grad_tile =
// dkappa' (Born), the second history (adjoint, 4-D) or A(mu^{m+1}) (Born-adjoint). cm/cp: the
// field's own memory-variable set (forward layout for the Born field, adjoint layout otherwise).
cudaError_t launch_so_step_cpml(int radius, int kind, const StepMaps &tm, const CpmlMaps &cm, const StepParams &p,
                                const CpmlParams &cp, const SoParams &q, cudaStream_t st);
cudaError_t launch_so_step(int radius, int kind, bool vd, const SoMaps &tm, const StepParams &p, const SoParams &q,
                           cudaStream_t st);
// Second-order term before the fold: a += b - (v / C) g on the padded grid of every shot, with v
// and C edge-replicated into the absorbing layer.
cudaError_t launch_so_combine(float *a, const float *b, const float *g, const float *sos, const float *dsos, int S,
                              int n_tx, int Nx, int Nz, int P, int nzp, int pitch, long long slice, cudaStream_t st);
// Exact misfit HVP: dmu's receiver source dkappa'_r 2 (M - M_obs) + kappa'_r 2 (J v).
cudaError_t launch_hvp_source(const float *cd_sim, const float *cd_obs, const float *dcd, const float *kap,
                              const float *dkap, const int *rx_node, float *asrc2, int S, int n_tx, int n_rx, int nt,
                              long long slice, int pitch, cudaStream_t st);
// Compensated forward step (modes kFwdSample, kFwdSampleHist, kFwdHist; p.tile_z must be 32).
cudaError_t launch_comp_step(int radius, int mode, const CompMaps &tm, const StepParams &p, const CompParams &q,
                             cudaStream_t st);
// s_R: the factor that makes the central weights of order `order` integers (0 for other orders).
double comp_weight_scale(int order);
// S: the factor that makes the staggered weights of order `order` integers (0 for other orders).
double comp_stagger_scale(int order);
// Compensated variable-density step (modes kFwdSample, kFwdSampleHist, kFwdHist; p.tile_z 32).
cudaError_t launch_comp_vd_step(int radius, int mode, const CompVdMaps &tm, const StepParams &p, const CompParams &q,
                                cudaStream_t st);
// kq = rho kappa'-form / S^2 (hi + lo) and the low parts of the buoyancies, from SoS and density.
cudaError_t launch_setup_comp_vd(const float *sos, const float *density, float *kq_hi, float *kq_lo, float *bx_lo,
                                 float *bz_lo, int n_maps, int Nx, int Nz, int P, int nzp, int pitch, double dt_over_dx,
                                 double stagger_scale, double d0, double dt, const int2 *map_dims, cudaStream_t st);
// kq = kappa' / s_R on the padded grid (FP64, split into hi + lo), for the compensated step.
cudaError_t launch_setup_kq(const float *sos, float *kq_hi, float *kq_lo, int n_maps, int Nx, int Nz, int P, int nzp,
                            int pitch, double dt_over_dx, double weight_scale, double d0, double dt,
                            const int2 *map_dims, cudaStream_t st);
// kappa' on the padded grid; with a density map kappa' = rho C^2 dt^2/(dx^2 (1 + D dt)), and the
// buoyancies bx, bz are written too (both may be null without a density map).
// unit_b: no density map, but buoyancies of 1 between nodes are written (staggered operator
// at constant density, used by the CPML).
cudaError_t launch_setup_kappa(const float *sos, const float *density, float *kap, float *bx, float *bz,
                               int *status, int n_maps, int Nx, int Nz, int P, int nxp, int nzp, int pitch,
                               double dt_over_dx, double d0, double dt, double c_max,
                               const int2 *map_dims, bool unit_b, cudaStream_t st);
cudaError_t launch_sample(const float *field, const int *rx_node, float *cd, long long slice,
                          int pitch, int S, int n_tx, int n_rx, int nt, int step, cudaStream_t st);
// cd_lo: low parts of the simulated traces (compensated forward steps), or null.
cudaError_t launch_residual(const float *cd_sim, const float *cd_lo, const float *cd_obs, const float *kap,
                            const int *rx_node, float *asrc, double *partial, int *status,
                            int S, int n_tx, int n_rx, int nt, long long slice, int pitch,
                            cudaStream_t st);
// dkappa' = kappa' * 2 dC / C on the padded grid (dC extended by edge replication).
cudaError_t launch_setup_dkappa(const float *sos, const float *dsos, const float *kap, float *dkap, int n_maps, int Nx,
                                int Nz, int P, int nzp, int pitch, cudaStream_t st);
cudaError_t launch_cotangent_source(const float *cd_grad, const float *kap, const int *rx_node, float *asrc,
                                   int *status, int S, int n_tx, int n_rx, int nt, long long slice, int pitch,
                                   cudaStream_t st);
cudaError_t launch_misfit_sum(const double *partial, double *misfit, int n_maps, int n_tx,
                              cudaStream_t st);
// grad64 (when not null) receives the gradient in FP64 instead of grad (FP32).
cudaError_t launch_fold(const float *g_shot, const float *sos, float *grad, double *grad64, double *fx, int n_maps,
                        int n_tx, int Nx, int Nz, int P, long long slice, int pitch, const int2 *map_dims,
                        cudaStream_t st);
cudaError_t launch_snap_absmax(const float *cur, const float *prev, unsigned *scale_bits, int S,
                               long long slice, int nxp, int nzp, int pitch, cudaStream_t st);
cudaError_t launch_snap_store(const float *cur, const float *prev, void *snap_u, void *snap_d,
                              const unsigned *scale_bits, int dtype, int S, long long slice,
                              int nxp, int nzp, int pitch, cudaStream_t st);
cudaError_t launch_snap_load(float *cur, float *prev, const void *snap_u, const void *snap_d,
                             const unsigned *scale_bits, int dtype, int S, long long slice,
                             int nxp, int nzp, int pitch, cudaStream_t st);

// Body of dufwi_simulate_sized. allow_groups false keeps every launch on the caller's stream
// (no group streams or events are created: the workspace-free entry point allocates nothing).
int simulate_impl(const dufwi_problem *pb, const dufwi_map_sizes *sizes, const float *sos, const float *density,
                  const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots, int n_maps, float *cd,
                  void *workspace, size_t workspace_bytes, void *stream, bool allow_groups);

}  // namespace dufwi
