/*
 * dufwi.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot path of deep-unfolded
 * full waveform inversion (DUFWI, arXiv 2603.04070). The library provides:
 *   - the time-domain damped acoustic simulation of transducer channel data (Sec. II-A, Eqs. 1-4);
 *   - the misfit of that simulation against observed data and its gradient with respect to the
 *     speed-of-sound (SoS) map (Sec. II-B, Eqs. 5-6). Every unfolded iteration consumes this
 *     gradient (Sec. III-A, Eq. 9).
 *
 * Conventions shared by every entry point:
 *   - Grids are row-major [z][x], x contiguous. The SoS map covers the physical grid nz x nx.
 *     The library adds `pml_cells` absorbing cells on every side internally, and extends the
 *     SoS into that layer by edge replication.
 *   - A "shot" is one (map, transmit) pair. Shots of map b are b*n_tx .. b*n_tx + n_tx - 1.
 *   - Channel data (CD) follow Eq. 3: M[p] is nt x n_rx, with M[p][t][r] the field U[t] at
 *     receiver r of transmit p, for t = 0..nt-1. U[0] = U[-1] = 0, so M[p][0][r] = 0.
 *   - Device arrays are caller-owned device pointers. Geometry tables are host pointers, which
 *     the library copies into the workspace with stream-ordered copies. The library allocates
 *     no memory: callers query the workspace size first and pass a device buffer at least that
 *     large, aligned to 256 bytes.
 *   - With the option DUFWI_OPT_REUSE_TABLES set, the library remembers, per workspace
 *     pointer, what it last copied there. A call on the same workspace with unchanged problem
 *     and geometry then skips those copies and issues only kernels, memsets and
 *     device-to-device copies, so it can be captured in a CUDA graph. Run it once outside the
 *     capture first. While the option is set, the workspace must stay reserved for the library
 *     between calls: a buffer freed and re-allocated at the same address would otherwise hold
 *     stale tables. Every index the kernels derive from the tables is bounds-checked, so
 *     damaged tables set DUFWI_ERR_GEOMETRY in the status word rather than touching memory
 *     outside the buffers.
 *   - Every call is asynchronous on the given stream and returns a status code. Host-side
 *     argument checks are reported by the return value. Conditions only visible on the device
 *     are recorded in a status word inside the workspace and read with dufwi_workspace_status:
 *       * an SoS value that is not finite, or not in (0, c_max];
 *       * non-finite observed data;
 *       * a density value that is not finite or not positive;
 *       * a bounded device wait that ran out.
 *     No C++ exception crosses this boundary.
 */
#ifndef DUFWI_H
#define DUFWI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define DUFWI_OK                 0
#define DUFWI_ERR_INVALID_ARG    1  /* a size, pointer or option is out of range */
#define DUFWI_ERR_CFL            2  /* c_max dt/dx above the stencil's stability limit, or SoS > c_max */
#define DUFWI_ERR_GEOMETRY       3  /* an element lies outside the physical grid */
#define DUFWI_ERR_UNSUPPORTED    4  /* a combination the library does not provide (see each call) */
#define DUFWI_ERR_WORKSPACE      5  /* workspace too small or misaligned */
#define DUFWI_ERR_CUDA           6  /* a CUDA runtime call failed */
#define DUFWI_ERR_TIMEOUT        7  /* a bounded device wait gave up */
#define DUFWI_ERR_NONFINITE      8  /* NaN/Inf in the SoS map or in the observed data */

/* Storage type of the checkpoint snapshots used by dufwi_misfit_gradient. Compressed snapshots
 * change the gradient only through the recomputed history (traces and misfit come from the first
 * sweep). Measured against the FP64 oracle on a cropped 256 x 256, 8-transmit, 3500-step case with
 * checkpoints every 100 steps: FP32 3.0e-5, FP16 5.5e-5, BF16 1.9e-4 (gradient rel-L2). FP16 stays
 * within the 1e-4 gradient bound of the FP32 path there; BF16 does not, and is offered for its
 * memory only (its 8-bit mantissa leaves ~4e-3 relative noise per stored value). */
#define DUFWI_SNAP_FP32 0           /* (U[t], U[t-1]) in FP32, exact */
#define DUFWI_SNAP_BF16 1           /* (U[t], U[t]-U[t-1]) in BF16, each scaled by its max |.|: outside the 1e-4 bound */
#define DUFWI_SNAP_FP16 2           /* (U[t], U[t]-U[t-1]) in FP16, each scaled by its max |.| */

/* Problem description: grid, time axis, absorbing layer, stencil, checkpointing.
 * Eq. 2 (Sec. II-A) is advanced with the coefficient maps
 *   a = (2 - D^2 dt^2)/(1 + D dt),  b = (D dt - 1)/(1 + D dt),  kappa = C^2 dt^2/(1 + D dt),
 * and the Laplacian is the central stencil of order fd_order divided by dx^2. The damping is
 * D(x,z) = d(xi_x) + d(xi_z), with d(xi) = d0 (xi/L)^2, L = pml_cells * dx, and
 * d0 = 3 pml_cref ln(1/pml_R) / (2L) (Sec. IV). */
typedef struct {
    int32_t nx, nz;          /* physical grid (cells), >= 1 each */
    double  dx, dt;          /* grid spacing (m) and time step (s), > 0 */
    int32_t nt;              /* recorded samples t = 0..nt-1, >= 1 */
    int32_t pml_cells;       /* absorbing cells per side, >= 1 (paper: 20) */
    double  pml_R;           /* target reflection factor in (0,1) (paper: 1e-3) */
    double  pml_cref;        /* reference SoS for d0, m/s (paper's water: 1500) */
    int32_t fd_order;        /* Laplacian order: 2, 4, 6 or 8 */
    int32_t snapshot_dtype;  /* DUFWI_SNAP_*; ignored by dufwi_simulate */
    int32_t ckpt_interval;   /* snapshot interval K in steps; 0 = keep every step (no recompute) */
    double  c_max;           /* upper bound of every SoS value (m/s), used for the CFL check */
    int32_t boundary;        /* DUFWI_BOUNDARY_*: absorbing layer of the pml_cells border cells */
    double  pml_alpha;       /* CPML only: frequency shift at the layer's inner edge (1/s), >= 0 */
    int32_t forward_precision; /* DUFWI_FORWARD_*: arithmetic of the forward (and recompute) steps */
    int32_t kept_segments;   /* gradient calls with checkpoints: how many of the last checkpoint
                              * segments keep their history from the forward sweep (at least the
                              * last one, which costs no memory: 0 and 1 are the same; >= the
                              * segment count = keep all, no snapshots) */
} dufwi_problem;

/* Hybrid history (kept_segments = k > 0 with ckpt_interval K > 0): the forward sweep writes the
 * history Lap(U^n) of the last k segments of K steps as it goes and takes snapshots only at the
 * starts of the earlier ones and of the first kept one (that one in FP32 whatever snapshot_dtype
 * says). The reverse sweep runs the adjoint straight through the kept
 * segments, then recomputes each earlier segment from its snapshot into the slots the kept
 * segments have freed. The history ring holds max(k, 1) segments, so the workspace grows by
 * (k - 1) K fields of S x (nz + 2P) x pitch floats, less the snapshots of the kept segments but
 * the first, and each kept segment saves one recompute of K steps. The last segment is always kept
 * (k >= 1): the ring holds one segment in any case. The reverse sweep recomputes the earlier
 * segments into the first kept segment's slots, so dufwi_backward recomputes that segment too,
 * from its snapshot: it can run any number of times after one dufwi_forward_save, while
 * dufwi_misfit_gradient uses the history its own forward sweep has just written. The results are
 * bit-identical to keeping every step (the recompute reproduces the forward sweep exactly with
 * FP32 snapshots).
 * dufwi_misfit, dufwi_jvp and the second-order calls ignore it. */

/* Arithmetic of the forward steps (the simulation of Eqs. 2-3, and the recompute of checkpoint
 * segments). The adjoint and the imaging condition run in FP32 in both modes.
 *   DUFWI_FORWARD_FP32: FP32 stencil and update; traces within ~1e-6 (rel-L2) of the FP64
 *     recursion. The gradient (Eq. 6) is linear in the residual r = M_sim - M_obs, so its error
 *     grows like |M| / |r|: 1e-3 to 1e-2 when a weak scatterer leaves r at 0.1-1 % of M.
 *   DUFWI_FORWARD_COMPENSATED: the field is carried as hi + lo FP32 planes and every rounding of
 *     the step is recovered with error-free transformations (TwoSum, TwoProd by FMA); the stencil
 *     weights are scaled to integers and kappa' and the damping coefficients are FP64 values held
 *     as hi + lo. Traces match the FP64 recursion to ~1e-13, and the residual is formed from
 *     (hi, lo) before rounding, so the gradient meets 1e-4 at any residual level. The traces
 *     returned are the hi planes (the FP32 rounding of the result). Costs: about 7x the FP32
 *     step's arithmetic, two more field planes and 8 B/cell more traffic per forward step, and
 *     FP32 snapshots of four planes instead of two. With a density map the staggered operator of
 *     Eq. 1 is compensated the same way (integer staggered weights, buoyancies and kappa' as
 *     hi + lo; about 10x the FP32 variable-density step's arithmetic). With the CPML, dufwi_jvp,
 *     dufwi_second_order or dufwi_hvp it returns DUFWI_ERR_UNSUPPORTED. The launch options (tile
 *     height, two steps, persistent sweeps, multi-tile, register caps, cluster sweeps) do not
 *     apply: the compensated step runs one launch per step and shot group on 64 x 32 tiles. */
#define DUFWI_FORWARD_FP32 0
#define DUFWI_FORWARD_COMPENSATED 1

/* Absorbing layers (both over pml_cells cells, quadratic damping profile d = d0 (xi/L)^2 with
 * d0 = 3 pml_cref ln(1/pml_R) / (2 L)):
 *   DUFWI_BOUNDARY_DAMPING: the damping term D of Eq. 1 (2 D u_t + D^2 u), the paper's layer.
 *   DUFWI_BOUNDARY_CPML: a convolutional PML on the staggered operator: each first difference
 *     is stretched by 1/s, s = 1 + d/(alpha + i omega), through one memory variable per
 *     difference and axis (recursive convolution; alpha = pml_alpha (1 - xi/L)); no damping
 *     term. Supported by dufwi_simulate, dufwi_simulate_noalloc, dufwi_misfit,
 *     dufwi_forward_save/dufwi_backward, dufwi_misfit_gradient, dufwi_second_order, dufwi_hvp,
 *     with or without a density map and with any ckpt_interval: a checkpoint stores the four
 *     memory fields read at its step in FP32 beside (U^t, U^{t-1}) (and the Born field's beside
 *     dU in the second-order calls), and each adjoint field keeps its own memory variables;
 *     dufwi_jvp too (the Born field with its own memory variables). Not by the *_sized calls
 *     (DUFWI_ERR_UNSUPPORTED). */
#define DUFWI_BOUNDARY_DAMPING 0
#define DUFWI_BOUNDARY_CPML 1

/* Transducer elements: physical-grid node indices (host arrays of n_elem entries). Elements
 * are point sources/receivers at nodes (the paper's elements act as both, Sec. II-A). */
typedef struct {
    int32_t n_elem;
    const int32_t *ix;
    const int32_t *iz;
} dufwi_array;

/* Transmit/receive pattern shared by every map (host arrays). Sequential transmission
 * (Sec. II-A): transmit p fires element tx_elem[p]; elements rx_elem[p][0..n_rx-1] record.
 * The receive subset may change between transmits. wavelet_per_tx = 0: one pulse [nt] for
 * all transmits; 1: one pulse per transmit [n_tx][nt]. */
typedef struct {
    int32_t n_tx, n_rx;
    const int32_t *tx_elem;   /* [n_tx] */
    const int32_t *rx_elem;   /* [n_tx][n_rx] */
    int32_t wavelet_per_tx;
} dufwi_shots;

/* Bytes of workspace needed by dufwi_simulate for n_maps maps. */
int dufwi_simulate_workspace_size(const dufwi_problem *pb, const dufwi_shots *shots,
                                  int32_t n_maps, size_t *bytes);

/* Bytes of workspace needed by dufwi_misfit_gradient for n_maps maps. It counts the snapshots
 * (every ckpt_interval steps) and one segment of recomputed history. */
int dufwi_workspace_size(const dufwi_problem *pb, const dufwi_shots *shots, int32_t n_maps,
                         size_t *bytes);

/* Forward model, Eqs. 2-4: the channel data of every shot.
 *   sos      [n_maps][nz][nx] float, device, m/s
 *   density  NULL (constant density, as in the paper) or [n_maps][nz][nx] float, device,
 *            kg/m^3: Eq. 1's rho div(rho^-1 grad u) on a staggered grid (half-point
 *            buoyancies). The result does not depend on a constant density. A value that is
 *            not finite or not positive is recorded in the workspace status word.
 *   wavelet  [nt] or [n_tx][nt] float, device. The source adds dt^2 w[t]/dx^2 at the transmit
 *            node in the step that produces U[t+1].
 *   cd       [n_maps][n_tx][nt][n_rx] float, device, output (may be NULL when n_rx = 0)
 *   workspace: device, >= dufwi_simulate_workspace_size bytes. */
int dufwi_simulate(const dufwi_problem *pb, const float *sos, const float *density,
                   const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                   int32_t n_maps, float *cd, void *workspace, size_t workspace_bytes,
                   void *stream /* cudaStream_t */);

/* Misfit and gradient, Eqs. 5-6 with lambda = 0, per map b:
 *   J[b] = sum over transmits, samples and receivers of (M_sim - M_obs)^2 (FP64 sum)
 *   g[b] = dJ[b]/dC on the physical grid. This is the exact gradient of the discrete J: the
 *          discrete adjoint of Eq. 2, with the zero-lag imaging condition, reduced over
 *          transmits in FP64, with the absorbing layer folded onto the edge cells.
 *   cd_obs  [n_maps][n_tx][nt][n_rx] float, device (may be NULL when n_rx = 0)
 *   misfit  [n_maps] double, device, output
 *   grad    [n_maps][nz][nx] float, device, output
 *   cd_sim  NULL or [n_maps][n_tx][nt][n_rx] float, device, output (the simulated data)
 *   workspace: device, >= dufwi_workspace_size bytes. */
int dufwi_misfit_gradient(const dufwi_problem *pb, const float *sos, const float *density,
                          const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                          int32_t n_maps, const float *cd_obs, double *misfit, float *grad,
                          float *cd_sim, void *workspace, size_t workspace_bytes,
                          void *stream /* cudaStream_t */);

/* dufwi_misfit_gradient with the gradient written in FP64: grad is [n_maps][nz][nx] double. The
 * per-shot imaging sums are FP32 as always; the sum over transmits, the fold of the absorbing layer
 * and the 2/C scaling are FP64 in both calls, and this one skips the final rounding to FP32. A
 * caller that splits the transmits of a map across devices sums these partial gradients in FP64
 * (Eqs. 5-6 are sums over transmits) and rounds once at the end. Same support as
 * dufwi_misfit_gradient. */
int dufwi_misfit_gradient_fp64(const dufwi_problem *pb, const float *sos, const float *density,
                               const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                               int32_t n_maps, const float *cd_obs, double *misfit, double *grad,
                               float *cd_sim, void *workspace, size_t workspace_bytes,
                               void *stream /* cudaStream_t */);

/* Forward model that keeps what the adjoint needs: the same channel data as dufwi_simulate, plus
 * the snapshots (every ckpt_interval steps) or the whole history, stored in `workspace`. The
 * workspace must hold dufwi_workspace_size bytes. Pair it with dufwi_backward, which turns any
 * cotangent of the channel data into a gradient with respect to the SoS map. Those two calls
 * are the forward and the backward of a differentiable simulator (Eq. 3 as a map C -> M). */
int dufwi_forward_save(const dufwi_problem *pb, const float *sos, const float *density,
                       const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                       int32_t n_maps, float *cd, void *workspace, size_t workspace_bytes,
                       void *stream /* cudaStream_t */);

/* Misfit only (Eq. 5 data term), without the gradient: one forward sweep per shot, then the
 * residual and the FP64 sum, exactly as in dufwi_misfit_gradient. It stores no snapshots and runs
 * no adjoint, so it costs about a third of a gradient. Line searches of a classical FWI loop
 * (Eq. 7) call it once per trial step.
 *   cd_obs  [n_maps][n_tx][nt][n_rx] float, device
 *   misfit  [n_maps] double, device, output: J_b = sum (M_sim - M_obs)^2
 *   cd_sim  NULL or [n_maps][n_tx][nt][n_rx] float, device, output
 *   workspace: device, >= dufwi_workspace_size bytes (the gradient's workspace).
 * For the same inputs J is bit-identical to the one dufwi_misfit_gradient returns. */
int dufwi_misfit(const dufwi_problem *pb, const float *sos, const float *density, const dufwi_array *arr,
                 const float *wavelet, const dufwi_shots *shots, int32_t n_maps, const float *cd_obs,
                 double *misfit, float *cd_sim, void *workspace, size_t workspace_bytes,
                 void *stream /* cudaStream_t */);

/* Vector-Jacobian product of the forward model: grad[b] = (dM[b]/dC[b])^T cd_grad[b] for each map.
 *   cd_grad  [n_maps][n_tx][nt][n_rx] float, device: the cotangent dL/dM
 *   grad     [n_maps][nz][nx] float, device, output
 * The call runs the discrete adjoint of Eq. 2, recomputing checkpoint segments from the
 * snapshots. It needs the workspace of a preceding dufwi_forward_save with the same problem,
 * maps, pulse and geometry, not overwritten in between. With cd_grad = 2 (M - M_obs) it gives
 * the gradient of dufwi_misfit_gradient, bit for bit. */
int dufwi_backward(const dufwi_problem *pb, const float *sos, const float *density,
                   const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                   int32_t n_maps, const float *cd_grad, float *grad, void *workspace,
                   size_t workspace_bytes, void *stream /* cudaStream_t */);

/* Jacobian-vector product of the forward model (the linearised, "Born" simulation): for a
 * perturbation dsos of the SoS maps, dcd[b] = (dM[b]/dC[b]) dsos[b]. Each time step advances the
 * background field (Eq. 2, recording the channel data into cd when cd is not NULL) and then the
 * perturbation field dU with the same update plus the source dkappa' Lap(U^n). Here
 * dkappa' = 2 kappa' dC / C, with dC extended into the absorbing layer like C. With
 * dufwi_backward this gives Gauss-Newton Hessian-vector products of the misfit,
 * H v = 2 J^T (J v). With a density map both fields use the variable-density operator and
 * Lap is that operator; with DUFWI_BOUNDARY_CPML Lap is the stretched operator G of the CPML
 * step and dU has memory variables of its own.
 *   dsos   [n_maps][nz][nx] float, device
 *   dcd    [n_maps][n_tx][nt][n_rx] float, device, output
 *   cd     NULL or [n_maps][n_tx][nt][n_rx] float, device, output (the background data)
 *   workspace: device, >= dufwi_jvp_workspace_size bytes. */
int dufwi_jvp_workspace_size(const dufwi_problem *pb, const dufwi_shots *shots, int32_t n_maps,
                             size_t *bytes);
int dufwi_jvp(const dufwi_problem *pb, const float *sos, const float *density, const dufwi_array *arr,
              const float *wavelet, const dufwi_shots *shots, int32_t n_maps, const float *dsos,
              float *dcd, float *cd, void *workspace, size_t workspace_bytes,
              void *stream /* cudaStream_t */);

/* Second-order product of the forward model: the derivative of the vector-Jacobian product
 * G = (dM/dC)^T cd_grad along an SoS direction dsos, with cd_grad held fixed,
 *   so[b] = d/dC[(dM[b]/dC[b])^T cd_grad[b]] . dsos[b]
 * (the Hessian of the scalar <M, cd_grad> applied to dsos). With cd_grad = 2 (M - M_obs) the
 * exact Hessian-vector product of the misfit (Eqs. 5-6) is H v = so + 2 J^T (J v), J = dM/dC;
 * the call returns J v as well (dcd). It differentiates the discrete adjoint once more: with
 * dkappa' = 2 kappa' dsos / C (dsos extended into the absorbing layer like C),
 *   dU^{n+1} = Eq. 2 on dU + dkappa' Lap(U^n)                       (the Born field of dufwi_jvp)
 *   mu^m     = Eq. 2 on mu + kappa' cd_grad^m at the receivers      (the adjoint of dufwi_backward)
 *   dmu^m    = Eq. 2 on dmu + dkappa' Lap(mu^{m+1}) + dkappa' cd_grad^m at the receivers
 *   so = (2/C) fold[sum_m dmu^m Lap(U^{m-1}) + mu^m Lap(dU^{m-1})] - (2 dsos / C^2) fold[sum_m mu^m Lap(U^{m-1})]
 * The forward pass keeps Lap(U^n) and Lap(dU^n) for every step (ckpt_interval 0) or, with
 * checkpoints, FP32 snapshots of U and dU every ckpt_interval steps (snapshot_dtype is not used
 * here) and recomputes each segment's two histories during the reverse pass.
 *   cd_grad [n_maps][n_tx][nt][n_rx] float, device (NULL only when n_rx == 0)
 *   dsos    [n_maps][nz][nx] float, device
 *   dcd     NULL or [n_maps][n_tx][nt][n_rx] float, device, output: J dsos
 *   so      [n_maps][nz][nx] float, device, output
 *   grad    NULL or [n_maps][nz][nx] float, device, output: (dM/dC)^T cd_grad
 *   workspace: device, >= dufwi_second_order_workspace_size bytes.
 * With a density map all three fields use the staggered variable-density operator of Eq. 1 (the
 * operator is symmetric, so the adjoint kinds use it as they are). With DUFWI_BOUNDARY_CPML Lap is
 * the stretched operator G of the CPML step (memory variables included), each of U, dU, mu and
 * dmu has its own memory variables, and in the dmu recursion dkappa' multiplies mu's adjoint
 * operator term A(mu^{m+1}) (mu^m = 2 mu^{m+1} - mu^{m+2} + kappa' A); tiles away from the
 * layer run the staggered kernel. The compensated forward steps give DUFWI_ERR_UNSUPPORTED.
 * The launch options (tile height, two-step, persistent) do not apply: every step uses 64 x 32
 * tiles, one launch per step and shot group (two with the CPML: interior and layer tiles). */
int dufwi_second_order_workspace_size(const dufwi_problem *pb, const dufwi_shots *shots,
                                      int32_t n_maps, size_t *bytes);
int dufwi_second_order(const dufwi_problem *pb, const float *sos, const float *density,
                       const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                       int32_t n_maps, const float *cd_grad, const float *dsos, float *dcd, float *so,
                       float *grad, void *workspace, size_t workspace_bytes,
                       void *stream /* cudaStream_t */);

/* Exact Hessian-vector product of the misfit J = sum (M - M_obs)^2 (Eqs. 5-6) in one call:
 *   hv[b] = H[b] dsos[b] = 2 J^T (J dsos) + d/dC[J^T w] . dsos,  w = 2 (M - M_obs), J = dM/dC,
 * with the misfit and its gradient beside it. It runs the sweeps of dufwi_second_order with
 * w known after the forward pass (the background traces are recorded). The adjoint of 2 J dsos
 * satisfies the same recursion as dmu, so it is carried by dmu through its receiver source
 * (dkappa'_r w + kappa'_r 2 (J dsos)) and shares dmu's imaging sum: no extra sweep.
 *   cd_obs [n_maps][n_tx][nt][n_rx] float, device (NULL only when n_rx == 0)
 *   dsos   [n_maps][nz][nx] float, device
 *   hv     [n_maps][nz][nx] float, device, output
 *   misfit NULL or [n_maps] double, device, output (as dufwi_misfit_gradient)
 *   grad   NULL or [n_maps][nz][nx] float, device, output (the misfit gradient)
 *   workspace: device, >= dufwi_second_order_workspace_size bytes.
 * Same support as dufwi_second_order. */
int dufwi_hvp(const dufwi_problem *pb, const float *sos, const float *density, const dufwi_array *arr,
              const float *wavelet, const dufwi_shots *shots, int32_t n_maps, const float *cd_obs,
              const float *dsos, float *hv, double *misfit, float *grad, void *workspace,
              size_t workspace_bytes, void *stream /* cudaStream_t */);

/* Forward model for callers that cannot allocate device memory. The paper has no counterpart:
 * this serves hosts that must not call cudaMalloc while running, such as a fixed-latency
 * acquisition loop (a device allocation can synchronise the device) or an application that hands
 * out all device memory from its own pool. The caller passes inputs and outputs as for
 * dufwi_simulate, but no workspace. The scratch space comes from one static device array of
 * DUFWI_NOALLOC_SCRATCH_BYTES inside the library. Every GPU that loads the library holds that
 * array until the process exits.
 *   - Size limit: problems whose dufwi_simulate_workspace_size exceeds the array are rejected with
 *     DUFWI_ERR_WORKSPACE before any device work.
 *   - First call on a device: it looks up the array's device address with that device current,
 *     then caches it. With lazy module loading (the CUDA default since 12.2) that lookup is also
 *     what loads the library's device code holding the array, so the first call on each device
 *     does reserve the array's memory and may synchronise. Make one warm-up call per device at
 *     start-up, before the phase that must not allocate and before any stream capture.
 *   - Sharing: all calls share the array, which keeps the last call's contents. Every buffer that
 *     must start at zero is cleared by the call itself. Calls that overlap on the GPU (other
 *     streams or host threads without ordering between them) race on the array.
 *   - Device-side conditions (an SoS value that is not finite or above c_max, an invalid density,
 *     a bounded wait that ran out) land in the status word at the start of the array, as they do
 *     in a caller's workspace; dufwi_noalloc_status reads it.
 * The call allocates no device memory: no cudaMalloc, no cudaFree, no allocating library call. */
#define DUFWI_NOALLOC_SCRATCH_BYTES (64u << 20)
int dufwi_simulate_noalloc(const dufwi_problem *pb, const float *sos, const float *density,
                           const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                           int32_t n_maps, float *cd, void *stream /* cudaStream_t */);

/* Device status of the last dufwi_simulate_noalloc call on the current device (the counterpart of
 * dufwi_workspace_status for the static array; the paper has none). It copies the status word
 * into host memory on `stream` and synchronises that stream, so call it after the simulation,
 * on the same stream. Returns the DUFWI_* code recorded by the kernels (DUFWI_OK if none), or
 * DUFWI_ERR_CUDA if the copy fails. It allocates nothing. */
int dufwi_noalloc_status(void *stream /* cudaStream_t */);

/* Maps of different sizes in one call (batching of uneven grids, Eq. 4 over many maps). The
 * problem's nx, nz define an envelope. Map b has its own physical grid nz[b] x nx[b] (1 <= nx[b]
 * <= nx, 1 <= nz[b] <= nz), with its own absorbing layer around it. Its SoS values fill the
 * leading nz[b] x nx[b] block of its slab in sos[n_maps][nz][nx]; the rest of the slab is
 * ignored. The gradient is written in the same layout, zero outside each map. Every element
 * named by the transmit/receive tables must lie inside every map. All shots of all maps advance
 * in the same launch per time step; tiles outside a map's padded grid exit at once. Workspace
 * sizes are those of the envelope (dufwi_simulate_workspace_size / dufwi_workspace_size).
 * The host arrays nx, nz hold n_maps entries each. */
typedef struct {
    const int32_t *nx;
    const int32_t *nz;
} dufwi_map_sizes;

int dufwi_simulate_sized(const dufwi_problem *pb, const dufwi_map_sizes *sizes, const float *sos,
                         const float *density, const dufwi_array *arr, const float *wavelet,
                         const dufwi_shots *shots, int32_t n_maps, float *cd, void *workspace,
                         size_t workspace_bytes, void *stream /* cudaStream_t */);

int dufwi_misfit_gradient_sized(const dufwi_problem *pb, const dufwi_map_sizes *sizes, const float *sos,
                                const float *density, const dufwi_array *arr, const float *wavelet,
                                const dufwi_shots *shots, int32_t n_maps, const float *cd_obs,
                                double *misfit, float *grad, float *cd_sim, void *workspace,
                                size_t workspace_bytes, void *stream /* cudaStream_t */);

/* Waits for the stream, then returns the device-side status word of the last call that used
 * this workspace (DUFWI_OK if none was raised). */
int dufwi_workspace_status(const void *workspace, void *stream /* cudaStream_t */);

/* Human-readable name of a status code (static storage). */
const char *dufwi_status_string(int status);

/* Largest stable c_max*dt/dx of the leapfrog scheme with the fd_order stencil in 2-D:
 * 2/sqrt(2 rho), rho = -(c_0 + 2 sum_k (-1)^k c_k) the magnitude of the 1-D stencil at the
 * Nyquist wavenumber. Returns a negative value for an unsupported order. */
double dufwi_cfl_limit(int32_t fd_order);

/* Sweep timing for measurement tools. While enabled, each call records CUDA events on its stream
 * around every sweep: the first forward sweep, each recompute segment, each adjoint segment, and
 * the remaining setup/residual/fold kernels. dufwi_profile_enable(1) creates a fixed pool of
 * events on the current device (outside any hot path); dufwi_profile_enable(0) destroys it.
 * dufwi_profile_read waits for the last recorded event, then writes the accumulated time (ms)
 * and the kernel launches per kind into ms[4] and launches[4]:
 *   0 forward sweep, 1 recompute, 2 adjoint, 3 other.
 * reset != 0 clears the accumulators. Recording stops silently when the pool is exhausted,
 * and the function then returns DUFWI_ERR_WORKSPACE. */
int dufwi_profile_enable(int enable);
int dufwi_profile_read(double *ms, int64_t *launches, int reset);

/* Tuning options of the step kernels. They are process-wide and change speed, never results
 * beyond rounding order.
 *   DUFWI_OPT_TILE_Z: output tile height of the one-step kernel, 32 (default) or 64 rows of 64
 *     columns.
 *   DUFWI_OPT_TWO_STEP: 1 advances pairs of time steps (n, n+1 with n even) in one launch,
 *     bit-identical to one launch per step (0, the default, which measured faster on GB300).
 *   DUFWI_OPT_REUSE_TABLES: 1 lets calls skip re-copying unchanged geometry tables into a
 *     workspace that stays reserved between calls (see the conventions above); default 0.
 *   DUFWI_OPT_PERSISTENT: 1 runs each sweep segment (the forward sweep between snapshots, a
 *     recompute segment, an adjoint segment) as one cooperative launch whose CTAs stay resident
 *     and pass 64 x 32 tiles from step to step through per-tile counters in the workspace,
 *     instead of one launch per time step; bit-identical results. Not used with the two-step
 *     kernel, the Born step or a density map; 0 (the default) launches once per step. The
 *     counters rely on all CTAs of the launch being resident: do not run other kernels on the
 *     device at the same time (another stream, another process). If residency is lost the
 *     bounded waits end the launch with DUFWI_ERR_TIMEOUT in the status word.
 *   DUFWI_OPT_MULTI_TILE: 1 runs the one-step kernel in its multi-tile form: a grid of as many
 *     CTAs as the device holds at once, each walking 64 x 32 tiles of all shots with two
 *     shared-memory stages, so the loads of the next tile overlap the arithmetic of the current
 *     one; bit-identical to the one-tile-per-CTA form. Not used with the two-step or persistent
 *     kernels, a density map, the CPML or the compensated forward steps.
 *   DUFWI_OPT_EARLY_LOADS: 1 (default) lets a one-step launch request the operands that neither
 *     of the two previous launches wrote (U^{n-1}, kappa', the adjoint's history tile) before it
 *     waits for the previous launch (programmatic dependent launch); 0 requests everything after
 *     the wait. Same results either way.
 *   DUFWI_OPT_SHOT_GROUPS: 1 to 4 (default 2). A call's shots (maps x transmits) are split into
 *     this many groups of consecutive shots (at most one group per shot), and each range of time
 *     steps launches one kernel per group and step, each group on a stream of its own that forks
 *     from the caller's stream before the range and joins it after. Shots never exchange data, so
 *     the groups run independently: a group's next step starts while the other group's step
 *     drains, which fills the SMs that one launch per step leaves idle at its start and end. The
 *     results are bit-identical for every value. The group streams and their events are created
 *     on a host thread's first grouped call on a device and kept until the thread exits; while the
 *     caller's stream is being captured into a CUDA graph they are not created, so a call captured
 *     before any uncaptured call on that thread and device runs as one group (make one uncaptured
 *     call first to capture the grouped form). Creating them is a stream and event creation: make
 *     a thread's first call outside another thread's global-mode stream capture. Not used with the two-step, persistent or
 *     multi-tile forms, or by dufwi_simulate_noalloc.
 *   DUFWI_OPT_MIN_CTAS: 4, 5 (default) or 6 resident CTAs per SM that the one-step kernel's
 *     register allocation is compiled for (96 registers at 5; 128 at 4; 80 at 6, with a few
 *     spills), for the 8th-order stencil with 64 x 32 tiles; other orders and tile heights use
 *     the build default. Same results for every value.
 *   DUFWI_OPT_CLUSTER: 1 runs each range of time steps (a sweep segment) of the compact
 *     stencil as one launch of one thread-block cluster of 8 CTAs per shot when the padded grid
 *     fits the cluster's shared memory (about 300 x 250 padded cells at most; each CTA holds a
 *     strip of rows and exchanges 4 halo rows per step with its neighbours through distributed
 *     shared memory, one cluster barrier per step), instead of one launch per step;
 *     bit-identical results. On GB300 it measured slower than one launch per step with
 *     programmatic dependent launch on the 128 x 128 and 188 x 188 workloads; it is an
 *     autotuner candidate. Not used
 *     with a density map, the CPML, the compensated steps, the Born and second-order calls, the
 *     *_sized calls or the two-step, persistent and multi-tile forms; 0 (default) otherwise.
 *   DUFWI_OPT_TEST_STALL: test hook for the bounded waits. 1 makes the next persistent sweep
 *     wait on a tile counter that nothing sets; that wait gives up after its time limit (2 s),
 *     the launch ends early with DUFWI_ERR_TIMEOUT in the workspace status word, and the device
 *     stays usable. The hook clears itself when used; 0 (default) disarms it.
 * Both functions return DUFWI_ERR_INVALID_ARG for an unknown option or value. */
#define DUFWI_OPT_TILE_Z 1
#define DUFWI_OPT_TWO_STEP 2
#define DUFWI_OPT_REUSE_TABLES 3
#define DUFWI_OPT_PERSISTENT 4
#define DUFWI_OPT_TEST_STALL 5
#define DUFWI_OPT_MULTI_TILE 6
#define DUFWI_OPT_EARLY_LOADS 7
#define DUFWI_OPT_SHOT_GROUPS 8
#define DUFWI_OPT_MIN_CTAS 9
#define DUFWI_OPT_CLUSTER 10
int dufwi_set_option(int32_t option, int32_t value);
int dufwi_get_option(int32_t option, int32_t *value);

/* Number of kernels this library has launched since it was loaded (all devices, all calls). */
int64_t dufwi_launch_count(void);

/* Library version, e.g. 0x000100 for 0.1.0. */
int32_t dufwi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DUFWI_H */
