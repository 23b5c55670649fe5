// dufwi_capi.cu -- host side of the C ABI declared in include/dufwi.h: argument validation,
// workspace layout, tensor-map construction and the launch sequence of the forward, recompute
// and adjoint sweeps. No allocation happens here; every buffer is carved out of the caller's
// workspace.
#include <math.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "../../include/dufwi.h"
#include "dufwi_internal.h"

namespace dufwi {
namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Central second-difference weights of Sec. II-A's Laplacian kernel (textbook values).
bool stencil_weights(int order, float c[5])
{
    for (int i = 0; i < 5; ++i) c[i] = 0.f;
    switch (order) {
    case 2: c[0] = -2.0f; c[1] = 1.0f; return true;
    case 4: c[0] = (float)(-5.0 / 2.0); c[1] = (float)(4.0 / 3.0); c[2] = (float)(-1.0 / 12.0); return true;
    case 6:
        c[0] = (float)(-49.0 / 18.0); c[1] = (float)(3.0 / 2.0); c[2] = (float)(-3.0 / 20.0);
        c[3] = (float)(1.0 / 90.0);
        return true;
    case 8:
        c[0] = (float)(-205.0 / 72.0); c[1] = (float)(8.0 / 5.0); c[2] = (float)(-1.0 / 5.0);
        c[3] = (float)(8.0 / 315.0); c[4] = (float)(-1.0 / 560.0);
        return true;
    default: return false;
    }
}

double stability_limit(int order)
{
    static const double w[4][5] = {{-2.0, 1.0, 0, 0, 0},
                                   {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0, 0, 0},
                                   {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0, 0},
                                   {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0}};
    if (order != 2 && order != 4 && order != 6 && order != 8) return -1.0;
    const double *c = w[order / 2 - 1];
    double nyq = c[0];
    for (int k = 1; k <= order / 2; ++k) nyq += 2.0 * c[k] * ((k & 1) ? -1.0 : 1.0);
    return 2.0 / sqrt(2.0 * fabs(nyq));
}

struct Layout {
    int Nx, Nz, P, nxp, nzp, pitch, radius, S, n_tx, n_rx, n_maps, nt, K, n_seg, n_hist;
    long long slice;
    size_t snap_elem;
    // byte offsets into the workspace
    size_t o_status, o_tx, o_rx, o_rxtab, o_rxsorted, o_damp, o_fold, o_kap, o_fa, o_fb, o_ma, o_mb, o_grad, o_hist, o_snap, o_scale, o_cd, o_asrc,
        o_part, total;
};

int validate_problem(const dufwi_problem *pb)
{
    if (!pb) return DUFWI_ERR_INVALID_ARG;
    float c[5];
    if (pb->nx < 1 || pb->nz < 1 || pb->nt < 1 || pb->pml_cells < 1) return DUFWI_ERR_INVALID_ARG;
    if (!(pb->dx > 0) || !(pb->dt > 0) || !(pb->pml_R > 0 && pb->pml_R < 1) || !(pb->pml_cref > 0))
        return DUFWI_ERR_INVALID_ARG;
    if (!stencil_weights(pb->fd_order, c)) return DUFWI_ERR_INVALID_ARG;
    if (pb->snapshot_dtype < DUFWI_SNAP_FP32 || pb->snapshot_dtype > DUFWI_SNAP_FP16) return DUFWI_ERR_INVALID_ARG;
    if (pb->ckpt_interval < 0) return DUFWI_ERR_INVALID_ARG;
    if (!(pb->c_max > 0) || !isfinite(pb->c_max)) return DUFWI_ERR_INVALID_ARG;
    if ((long long)pb->nx + 2LL * pb->pml_cells > 65535 || (long long)pb->nz + 2LL * pb->pml_cells > 65535)
        return DUFWI_ERR_INVALID_ARG;
    if (pb->c_max * pb->dt / pb->dx > stability_limit(pb->fd_order)) return DUFWI_ERR_CFL;
    return DUFWI_OK;
}

int make_layout(const dufwi_problem *pb, const dufwi_shots *sh, int n_maps, bool gradient, Layout *L)
{
    int rc = validate_problem(pb);
    if (rc) return rc;
    if (!sh || sh->n_tx < 1 || sh->n_rx < 0 || n_maps < 1) return DUFWI_ERR_INVALID_ARG;
    if (sh->wavelet_per_tx != 0 && sh->wavelet_per_tx != 1) return DUFWI_ERR_INVALID_ARG;
    memset(L, 0, sizeof(*L));
    L->Nx = pb->nx; L->Nz = pb->nz; L->P = pb->pml_cells;
    L->nxp = pb->nx + 2 * pb->pml_cells;
    L->nzp = pb->nz + 2 * pb->pml_cells;
    L->pitch = (L->nxp + 7) / 8 * 8;
    L->slice = (long long)L->nzp * L->pitch;
    L->radius = pb->fd_order / 2;
    L->n_tx = sh->n_tx; L->n_rx = sh->n_rx; L->n_maps = n_maps; L->nt = pb->nt;
    L->S = n_maps * sh->n_tx;
    if ((long long)n_maps * sh->n_tx > 65535) return DUFWI_ERR_INVALID_ARG;   // grid.z limit
    const int steps = pb->nt - 1;
    if (pb->ckpt_interval == 0 || pb->ckpt_interval >= steps) {
        L->K = steps > 0 ? steps : 1;
        L->n_seg = 1;
    } else {
        L->K = pb->ckpt_interval;
        L->n_seg = (steps + L->K - 1) / L->K;
    }
    L->n_hist = (pb->ckpt_interval == 0) ? (steps > 0 ? steps : 1) : L->K;
    L->snap_elem = pb->snapshot_dtype == DUFWI_SNAP_FP32 ? 4 : 2;

    const size_t field = (size_t)L->S * L->slice * sizeof(float);
    const size_t cdb = (size_t)L->S * L->nt * (L->n_rx > 0 ? L->n_rx : 1) * sizeof(float);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, kAlign); return o; };
    L->o_status = take(sizeof(int));
    L->o_tx = take(sizeof(int) * L->n_tx);
    L->o_rx = take(sizeof(int) * (size_t)L->n_tx * (L->n_rx > 0 ? L->n_rx : 1));
    const size_t tiles_max = (size_t)((L->nxp + kTileX - 1) / kTileX) * ((L->nzp + 31) / 32);
    L->o_rxtab = take(sizeof(int2) * (size_t)L->n_tx * tiles_max);
    L->o_rxsorted = take(sizeof(int) * (size_t)L->n_tx * (L->n_rx > 0 ? L->n_rx : 1));
    L->o_damp = take(sizeof(float2) * (size_t)(L->P + 1) * (L->P + 1));
    L->o_kap = take((size_t)n_maps * L->slice * sizeof(float));
    L->o_fa = take(field);
    L->o_fb = take(field);
    if (gradient) {
        const bool store_all = pb->ckpt_interval == 0 || pb->ckpt_interval >= steps;
        L->o_ma = take(field);
        L->o_mb = take(field);
        L->o_grad = take(field);
        L->o_hist = take(field * (size_t)L->n_hist);
        if (!store_all) {
            L->o_snap = take((size_t)L->n_seg * 2 * L->S * L->slice * L->snap_elem);
            L->o_scale = take((size_t)L->n_seg * 2 * L->S * sizeof(unsigned));
        }
        L->o_cd = take(cdb);
        L->o_asrc = take(cdb);
        L->o_part = take((size_t)L->S * sizeof(double));
        L->o_fold = take((size_t)n_maps * L->nzp * L->Nx * sizeof(double));
    }
    L->total = off;
    return DUFWI_OK;
}

int check_geometry(const dufwi_array *arr, const dufwi_shots *sh, const Layout &L, std::vector<int> &tx,
                   std::vector<int> &rx)
{
    if (!arr || !arr->ix || !arr->iz || arr->n_elem < 1 || !sh->tx_elem || (sh->n_rx > 0 && !sh->rx_elem))
        return DUFWI_ERR_INVALID_ARG;
    auto node = [&](int e, int *out) {
        if (e < 0 || e >= arr->n_elem) return DUFWI_ERR_GEOMETRY;
        const int ix = arr->ix[e], iz = arr->iz[e];
        if (ix < 0 || ix >= L.Nx || iz < 0 || iz >= L.Nz) return DUFWI_ERR_GEOMETRY;
        *out = ((iz + L.P) << 16) | (ix + L.P);
        return DUFWI_OK;
    };
    tx.assign(L.n_tx, 0);
    rx.assign((size_t)L.n_tx * (L.n_rx > 0 ? L.n_rx : 1), 0);
    for (int t = 0; t < L.n_tx; ++t) {
        int rc = node(sh->tx_elem[t], &tx[t]);
        if (rc) return rc;
        for (int r = 0; r < L.n_rx; ++r) {
            rc = node(sh->rx_elem[(size_t)t * L.n_rx + r], &rx[(size_t)t * L.n_rx + r]);
            if (rc) return rc;
        }
    }
    return DUFWI_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// FP32 tensor map of rank 3 or 4 over a [..][nzp][pitch] buffer: dims (nxp, nzp, d2[, d3]),
// row stride pitch, slice stride nzp * pitch, box (bx, bz, 1[, 1]). Elements outside the tensor
// (x >= nxp, z < 0 or z >= nzp) read as zero, the stencil's zero exterior.
int tensor_map(CUtensorMap *tm, const void *base, const Layout &L, int d2, int d3, int bx, int bz)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return DUFWI_ERR_CUDA;
    const cuuint32_t rank = d3 > 0 ? 4 : 3;
    cuuint64_t dims[4] = {(cuuint64_t)L.nxp, (cuuint64_t)L.nzp, (cuuint64_t)d2, (cuuint64_t)(d3 > 0 ? d3 : 1)};
    cuuint64_t strides[3] = {(cuuint64_t)L.pitch * sizeof(float), (cuuint64_t)L.slice * sizeof(float),
                             (cuuint64_t)L.slice * sizeof(float) * (cuuint64_t)d2};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)bz, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? DUFWI_OK : DUFWI_ERR_CUDA;
}

// Tile height of the step kernels (DUFWI_OPT_TILE_Z).
int g_tile_z = kTileZDefault;

// Maps of a step that reads `cur` with halo and updates `out` in place (tile height tz).
int step_maps(StepMaps *m, const float *cur, const float *out, const float *kap, const float *hist, int n_hist,
              const float *grad, const Layout &L, int tz)
{
    memset(m, 0, sizeof(*m));
    int rc = tensor_map(&m->cur_box, cur, L, L.S, 0, kBoxX, tz + 2 * kHalo);
    if (!rc) rc = tensor_map(&m->out_tile, out, L, L.S, 0, kTileX, tz);
    if (!rc) rc = tensor_map(&m->kap_tile, kap, L, L.n_maps, 0, kTileX, tz);
    if (!rc && hist) rc = tensor_map(&m->hist_tile, hist, L, L.S, n_hist, kTileX, tz);
    if (!rc && grad) rc = tensor_map(&m->grad_tile, grad, L, L.S, 0, kTileX, tz);
    return rc;
}

#define CK(x)                                                                                                        \
    do {                                                                                                             \
        if ((x) != cudaSuccess) return DUFWI_ERR_CUDA;                                                               \
    } while (0)

std::atomic<long long> g_launches{0};

// Checks a kernel launch and counts it (globally and in the caller's local counter `nl`).
#define CKL(x)                                                                                                       \
    do {                                                                                                             \
        if ((x) != cudaSuccess) return DUFWI_ERR_CUDA;                                                               \
        ++nl;                                                                                                        \
        g_launches.fetch_add(1, std::memory_order_relaxed);                                                          \
    } while (0)

// Event-based sweep timing (see dufwi_profile_enable).
struct Profiler {
    struct Span {
        int kind, e0, e1;
        long long launches;
    };
    bool on = false;
    bool overflow = false;
    int device = -1;
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    std::vector<Span> spans;
    double ms[4] = {0, 0, 0, 0};
    long long launches[4] = {0, 0, 0, 0};

    int mark(cudaStream_t st)
    {
        if (!on) return -1;
        if (next >= pool.size()) { overflow = true; return -1; }
        if (cudaEventRecord(pool[next], st) != cudaSuccess) return -1;
        return (int)next++;
    }
    void span(int kind, int e0, int e1, long long n)
    {
        if (e0 < 0 || e1 < 0) return;
        if (spans.size() < spans.capacity()) spans.push_back({kind, e0, e1, n});
        else overflow = true;
    }
};
Profiler g_prof;
constexpr size_t kProfEvents = 1 << 14;

struct Ctx {
    Layout L;
    const dufwi_problem *pb;
    char *ws;
    cudaStream_t st;
    StepParams base;
    int *status() const { return reinterpret_cast<int *>(ws + L.o_status); }
    template <typename T> T *at(size_t o) const { return reinterpret_cast<T *>(ws + o); }
};

int common_setup(Ctx &c, const float *sos, const float *density, const dufwi_array *arr, const float *wavelet,
                 const dufwi_shots *sh, void *workspace, size_t ws_bytes, void *stream, bool gradient)
{
    const Layout &L = c.L;
    if (!sos || !wavelet || !workspace) return DUFWI_ERR_INVALID_ARG;
    if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return DUFWI_ERR_WORKSPACE;
    std::vector<int> tx, rx;
    int rc = check_geometry(arr, sh, L, tx, rx);
    if (rc) return rc;
    c.ws = static_cast<char *>(workspace);
    c.st = static_cast<cudaStream_t>(stream);
    // receivers grouped by the step-kernel tile that contains them, per transmit
    const int tz = g_tile_z;
    const int tiles_x = (L.nxp + kTileX - 1) / kTileX, tiles = tiles_x * ((L.nzp + tz - 1) / tz);
    std::vector<int2> tab((size_t)L.n_tx * tiles, make_int2(0, 0));
    std::vector<int> sorted((size_t)L.n_tx * (L.n_rx > 0 ? L.n_rx : 1), 0);
    std::vector<int> tile_of(L.n_rx > 0 ? L.n_rx : 1);
    for (int t = 0; t < L.n_tx; ++t) {
        int2 *row = tab.data() + (size_t)t * tiles;
        for (int r = 0; r < L.n_rx; ++r) {
            const int node = rx[(size_t)t * L.n_rx + r];
            tile_of[r] = ((node >> 16) / tz) * tiles_x + (node & 0xffff) / kTileX;
            row[tile_of[r]].y++;
        }
        int acc = 0;
        for (int k = 0; k < tiles; ++k) { row[k].x = acc; acc += row[k].y; }
        std::vector<int> fill(tiles, 0);
        for (int r = 0; r < L.n_rx; ++r)
            sorted[(size_t)t * L.n_rx + row[tile_of[r]].x + fill[tile_of[r]]++] = r;
    }
    // damping terms (a - 2, b + 1) of Eq. 2 at every pair of layer depths, in FP64, rounded once
    const dufwi_problem *pbh = c.pb;
    const double d0h = 3.0 * pbh->pml_cref * log(1.0 / pbh->pml_R) / (2.0 * pbh->pml_cells * pbh->dx);
    std::vector<float2> damp((size_t)(L.P + 1) * (L.P + 1));
    for (int dz = 0; dz <= L.P; ++dz)
        for (int dxl = 0; dxl <= L.P; ++dxl) {
            const double xz = (double)dz / L.P, xx = (double)dxl / L.P;
            const double q = (d0h * xx * xx + d0h * xz * xz) * pbh->dt;
            damp[(size_t)dz * (L.P + 1) + dxl] = make_float2((float)(-q * (2.0 + q) / (1.0 + q)), (float)(2.0 * q / (1.0 + q)));
        }
    CK(cudaMemsetAsync(c.status(), 0, sizeof(int), c.st));
    CK(cudaMemcpyAsync(c.at<float2>(L.o_damp), damp.data(), sizeof(float2) * damp.size(), cudaMemcpyHostToDevice,
                       c.st));
    CK(cudaMemcpyAsync(c.at<int>(L.o_tx), tx.data(), sizeof(int) * tx.size(), cudaMemcpyHostToDevice, c.st));
    CK(cudaMemcpyAsync(c.at<int>(L.o_rx), rx.data(), sizeof(int) * rx.size(), cudaMemcpyHostToDevice, c.st));
    CK(cudaMemcpyAsync(c.at<int2>(L.o_rxtab), tab.data(), sizeof(int2) * tab.size(), cudaMemcpyHostToDevice, c.st));
    CK(cudaMemcpyAsync(c.at<int>(L.o_rxsorted), sorted.data(), sizeof(int) * sorted.size(), cudaMemcpyHostToDevice,
                       c.st));
    // copies from pageable memory are staged before cudaMemcpyAsync returns
    const dufwi_problem *pb = c.pb;
    const double d0 = 3.0 * pb->pml_cref * log(1.0 / pb->pml_R) / (2.0 * pb->pml_cells * pb->dx);
    long long nl = 0;
    const int e0 = g_prof.mark(c.st);
    CKL(launch_setup_kappa(sos, density, c.at<float>(L.o_kap), c.status(), L.n_maps, L.Nx, L.Nz, L.P, L.nxp, L.nzp,
                           L.pitch, pb->dt / pb->dx, d0, pb->dt, pb->c_max, c.st));
    g_prof.span(3, e0, g_prof.mark(c.st), nl);

    StepParams &p = c.base;
    memset(&p, 0, sizeof(p));
    p.kap = c.at<float>(L.o_kap);
    p.status = c.status();
    p.slice = L.slice;
    p.nxp = L.nxp; p.nzp = L.nzp; p.pitch = L.pitch;
    p.n_maps = L.n_maps; p.n_tx = L.n_tx; p.n_rx = L.n_rx; p.nt = L.nt;
    p.wav_per_tx = sh->wavelet_per_tx;
    p.inj_scale = (float)(pb->dt * pb->dt / (pb->dx * pb->dx));
    p.P = L.P; p.Nx = L.Nx; p.Nz = L.Nz;
    p.damp_tab = c.at<float2>(L.o_damp);
    stencil_weights(pb->fd_order, p.c);
    p.tile_z = tz;
    p.rx_tab = c.at<int2>(L.o_rxtab);
    p.rx_sorted = c.at<int>(L.o_rxsorted);
    (void)gradient;
    return DUFWI_OK;
}

// Forward sweep from rest over steps [0, nt-1): U^{n+1} from U^n and U^{n-1}, recording U^n at
// the receivers; optional history (store-all) and snapshots every K steps.
int forward_sweep(Ctx &c, const float *wavelet, float *cd, float *fa, float *fb, const StepMaps &ta,
                  const StepMaps &tb, bool store_hist, bool snapshots)
{
    const Layout &L = c.L;
    long long nl = 0;
    const int e0 = g_prof.mark(c.st);
    const size_t field = (size_t)L.S * L.slice * sizeof(float);
    CK(cudaMemsetAsync(fa, 0, field, c.st));
    CK(cudaMemsetAsync(fb, 0, field, c.st));
    float *cur = fa, *prv = fb;
    const StepMaps *tcur = &ta, *tprv = &tb;
    StepParams p = c.base;
    p.inj_node = c.at<int>(L.o_tx);
    p.inj_val = wavelet;
    p.smp_node = c.at<int>(L.o_rx);
    p.cd = cd;
    const int dtype = c.pb->snapshot_dtype;
    for (int n = 0; n < L.nt - 1; ++n) {
        if (snapshots && n % L.K == 0) {
            const int sg = n / L.K;
            char *snap = c.at<char>(L.o_snap) + (size_t)sg * 2 * L.S * L.slice * L.snap_elem;
            char *snap_d = snap + (size_t)L.S * L.slice * L.snap_elem;
            if (dtype == DUFWI_SNAP_FP32) {
                CK(cudaMemcpyAsync(snap, cur, field, cudaMemcpyDeviceToDevice, c.st));
                CK(cudaMemcpyAsync(snap_d, prv, field, cudaMemcpyDeviceToDevice, c.st));
            } else {
                unsigned *sc = c.at<unsigned>(L.o_scale) + (size_t)sg * 2 * L.S;
                CK(cudaMemsetAsync(sc, 0, 2 * L.S * sizeof(unsigned), c.st));
                CKL(launch_snap_absmax(cur, prv, sc, L.S, L.slice, L.nxp, L.nzp, L.pitch, c.st));
                CKL(launch_snap_store(cur, prv, snap, snap_d, sc, dtype, L.S, L.slice, L.nxp, L.nzp, L.pitch, c.st));
            }
        }
        p.out = prv;
        p.step = n;
        p.hist = store_hist ? c.at<float>(L.o_hist) + (size_t)n * L.S * L.slice : nullptr;
        CKL(launch_step(L.radius, store_hist ? kFwdSampleHist : kFwdSample, *tcur, p, c.st));
        float *t = cur; cur = prv; prv = t;
        const StepMaps *tt = tcur; tcur = tprv; tprv = tt;
    }
    if (L.n_rx > 0)
        CKL(launch_sample(cur, c.at<int>(L.o_rx), cd, L.slice, L.pitch, L.S, L.n_tx, L.n_rx, L.nt, L.nt - 1, c.st));
    g_prof.span(0, e0, g_prof.mark(c.st), nl);
    return DUFWI_OK;
}

}  // namespace
}  // namespace dufwi

using namespace dufwi;

extern "C" {

int32_t dufwi_version(void) { return 0x000100; }

int dufwi_set_option(int32_t option, int32_t value)
{
    switch (option) {
    case DUFWI_OPT_TILE_Z:
        if (value != 32 && value != 64) return DUFWI_ERR_INVALID_ARG;
        g_tile_z = value;
        return DUFWI_OK;
    default: return DUFWI_ERR_INVALID_ARG;
    }
}

int dufwi_get_option(int32_t option, int32_t *value)
{
    if (!value) return DUFWI_ERR_INVALID_ARG;
    switch (option) {
    case DUFWI_OPT_TILE_Z: *value = g_tile_z; return DUFWI_OK;
    default: return DUFWI_ERR_INVALID_ARG;
    }
}

int64_t dufwi_launch_count(void) { return (int64_t)g_launches.load(); }

int dufwi_profile_enable(int enable)
{
    if (enable && !g_prof.on) {
        if (g_prof.pool.empty()) {
            g_prof.pool.resize(kProfEvents);
            for (auto &e : g_prof.pool)
                if (cudaEventCreate(&e) != cudaSuccess) return DUFWI_ERR_CUDA;
            g_prof.spans.reserve(kProfEvents);
            if (cudaGetDevice(&g_prof.device) != cudaSuccess) return DUFWI_ERR_CUDA;
        }
        g_prof.on = true;
    } else if (!enable && g_prof.on) {
        g_prof.on = false;
        for (auto &e : g_prof.pool) cudaEventDestroy(e);
        g_prof.pool.clear();
        g_prof.spans.clear();
        g_prof.next = 0;
    }
    return DUFWI_OK;
}

int dufwi_profile_read(double *ms, int64_t *launches, int reset)
{
    if (!ms || !launches) return DUFWI_ERR_INVALID_ARG;
    if (g_prof.next > 0 && cudaEventSynchronize(g_prof.pool[g_prof.next - 1]) != cudaSuccess) return DUFWI_ERR_CUDA;
    for (const auto &sp : g_prof.spans) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g_prof.pool[sp.e0], g_prof.pool[sp.e1]) != cudaSuccess) return DUFWI_ERR_CUDA;
        g_prof.ms[sp.kind] += t;
        g_prof.launches[sp.kind] += sp.launches;
    }
    g_prof.spans.clear();
    g_prof.next = 0;
    for (int k = 0; k < 4; ++k) { ms[k] = g_prof.ms[k]; launches[k] = g_prof.launches[k]; }
    const bool ovf = g_prof.overflow;
    if (reset) {
        for (int k = 0; k < 4; ++k) { g_prof.ms[k] = 0; g_prof.launches[k] = 0; }
        g_prof.overflow = false;
    }
    return ovf ? DUFWI_ERR_WORKSPACE : DUFWI_OK;
}

double dufwi_cfl_limit(int32_t fd_order) { return stability_limit(fd_order); }

const char *dufwi_status_string(int status)
{
    switch (status) {
    case DUFWI_OK: return "ok";
    case DUFWI_ERR_INVALID_ARG: return "invalid argument";
    case DUFWI_ERR_CFL: return "CFL condition violated (or SoS above c_max)";
    case DUFWI_ERR_GEOMETRY: return "element outside the physical grid";
    case DUFWI_ERR_UNSUPPORTED: return "unsupported (non-constant density)";
    case DUFWI_ERR_WORKSPACE: return "workspace too small or misaligned";
    case DUFWI_ERR_CUDA: return "CUDA error";
    case DUFWI_ERR_TIMEOUT: return "device wait timed out";
    case DUFWI_ERR_NONFINITE: return "non-finite input";
    default: return "unknown status";
    }
}

int dufwi_simulate_workspace_size(const dufwi_problem *pb, const dufwi_shots *shots, int32_t n_maps, size_t *bytes)
{
    if (!bytes) return DUFWI_ERR_INVALID_ARG;
    Layout L;
    int rc = make_layout(pb, shots, n_maps, false, &L);
    if (rc) return rc;
    *bytes = L.total;
    return DUFWI_OK;
}

int dufwi_workspace_size(const dufwi_problem *pb, const dufwi_shots *shots, int32_t n_maps, size_t *bytes)
{
    if (!bytes) return DUFWI_ERR_INVALID_ARG;
    Layout L;
    int rc = make_layout(pb, shots, n_maps, true, &L);
    if (rc) return rc;
    *bytes = L.total;
    return DUFWI_OK;
}

int dufwi_workspace_status(const void *workspace, void *stream)
{
    if (!workspace) return DUFWI_ERR_INVALID_ARG;
    int h = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&h, workspace, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DUFWI_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DUFWI_ERR_CUDA;
    return h;
}

int dufwi_simulate(const dufwi_problem *pb, const float *sos, const float *density, const dufwi_array *arr,
                   const float *wavelet, const dufwi_shots *shots, int32_t n_maps, float *cd, void *workspace,
                   size_t workspace_bytes, void *stream)
{
    Ctx c;
    c.pb = pb;
    int rc = make_layout(pb, shots, n_maps, false, &c.L);
    if (rc) return rc;
    if (!cd && c.L.n_rx > 0) return DUFWI_ERR_INVALID_ARG;
    rc = common_setup(c, sos, density, arr, wavelet, shots, workspace, workspace_bytes, stream, false);
    if (rc) return rc;
    float *fa = c.at<float>(c.L.o_fa), *fb = c.at<float>(c.L.o_fb);
    const float *kap = c.at<float>(c.L.o_kap);
    StepMaps ta, tb;
    if (step_maps(&ta, fa, fb, kap, nullptr, 0, nullptr, c.L, c.base.tile_z) || step_maps(&tb, fb, fa, kap, nullptr, 0, nullptr, c.L, c.base.tile_z))
        return DUFWI_ERR_CUDA;
    return forward_sweep(c, wavelet, cd, fa, fb, ta, tb, false, false);
}

int dufwi_misfit_gradient(const dufwi_problem *pb, const float *sos, const float *density, const dufwi_array *arr,
                          const float *wavelet, const dufwi_shots *shots, int32_t n_maps, const float *cd_obs,
                          double *misfit, float *grad, float *cd_sim, void *workspace, size_t workspace_bytes,
                          void *stream)
{
    Ctx c;
    c.pb = pb;
    int rc = make_layout(pb, shots, n_maps, true, &c.L);
    if (rc) return rc;
    if ((!cd_obs && c.L.n_rx > 0) || !misfit || !grad) return DUFWI_ERR_INVALID_ARG;
    rc = common_setup(c, sos, density, arr, wavelet, shots, workspace, workspace_bytes, stream, true);
    if (rc) return rc;
    const Layout &L = c.L;
    const size_t field = (size_t)L.S * L.slice * sizeof(float);
    float *fa = c.at<float>(L.o_fa), *fb = c.at<float>(L.o_fb);
    float *ma = c.at<float>(L.o_ma), *mb = c.at<float>(L.o_mb);
    const float *kap = c.at<float>(L.o_kap);
    float *hist = c.at<float>(L.o_hist);
    float *g_shot = c.at<float>(L.o_grad);
    StepMaps ta, tb, tma, tmb;
    if (step_maps(&ta, fa, fb, kap, nullptr, 0, nullptr, L, c.base.tile_z) || step_maps(&tb, fb, fa, kap, nullptr, 0, nullptr, L, c.base.tile_z) ||
        step_maps(&tma, ma, mb, kap, hist, L.n_hist, g_shot, L, c.base.tile_z) || step_maps(&tmb, mb, ma, kap, hist, L.n_hist, g_shot, L, c.base.tile_z))
        return DUFWI_ERR_CUDA;
    const bool store_all = (L.n_seg == 1);
    float *cd = c.at<float>(L.o_cd);

    // 1. forward sweep: traces, and either the whole history or the snapshots
    rc = forward_sweep(c, wavelet, cd, fa, fb, ta, tb, store_all, !store_all);
    if (rc) return rc;
    if (cd_sim && L.n_rx > 0) CK(cudaMemcpyAsync(cd_sim, cd, (size_t)L.S * L.nt * L.n_rx * sizeof(float), cudaMemcpyDeviceToDevice, c.st));

    // 2. residual, misfit and adjoint source
    float *asrc = c.at<float>(L.o_asrc);
    double *part = c.at<double>(L.o_part);
    long long nl = 0;
    int e0 = g_prof.mark(c.st);
    CKL(launch_residual(cd, cd_obs, c.at<float>(L.o_kap), c.at<int>(L.o_rx), asrc, part, c.status(), L.S, L.n_tx,
                        L.n_rx, L.nt, L.slice, L.pitch, c.st));
    CKL(launch_misfit_sum(part, misfit, L.n_maps, L.n_tx, c.st));
    g_prof.span(3, e0, g_prof.mark(c.st), nl);

    // 3. reverse sweep, segment by segment
    CK(cudaMemsetAsync(ma, 0, field, c.st));
    CK(cudaMemsetAsync(mb, 0, field, c.st));
    CK(cudaMemsetAsync(g_shot, 0, field, c.st));
    float *mcur = ma, *mprv = mb;                 // mu^{m+1}, mu^{m+2}
    const StepMaps *tmc = &tma, *tmp = &tmb;
    StepParams ap = c.base;
    ap.inj_node = c.at<int>(L.o_rx);
    ap.inj_val = asrc;
    ap.grad = g_shot;
    StepParams fp = c.base;
    fp.inj_node = c.at<int>(L.o_tx);
    fp.inj_val = wavelet;
    const int dtype = pb->snapshot_dtype;
    const size_t hstride = (size_t)L.S * L.slice;
    for (int sg = L.n_seg - 1; sg >= 0; --sg) {
        const int t0 = store_all ? 0 : sg * L.K;
        const int t1 = store_all ? L.nt - 1 : (t0 + L.K < L.nt - 1 ? t0 + L.K : L.nt - 1);
        if (!store_all) {
            nl = 0;
            e0 = g_prof.mark(c.st);
            // restore (U^{t0}, U^{t0-1}) and recompute Lap(U^n) for n = t0 .. t1-1
            char *snap = c.at<char>(L.o_snap) + (size_t)sg * 2 * L.S * L.slice * L.snap_elem;
            char *snap_d = snap + (size_t)L.S * L.slice * L.snap_elem;
            if (dtype == DUFWI_SNAP_FP32) {
                CK(cudaMemcpyAsync(fa, snap, field, cudaMemcpyDeviceToDevice, c.st));
                CK(cudaMemcpyAsync(fb, snap_d, field, cudaMemcpyDeviceToDevice, c.st));
            } else {
                const unsigned *sc = c.at<unsigned>(L.o_scale) + (size_t)sg * 2 * L.S;
                CKL(launch_snap_load(fa, fb, snap, snap_d, sc, dtype, L.S, L.slice, L.nxp, L.nzp, L.pitch, c.st));
            }
            float *cur = fa, *prv = fb;
            const StepMaps *tc = &ta, *tp = &tb;
            for (int n = t0; n < t1; ++n) {
                fp.out = prv;
                fp.step = n;
                fp.hist = hist + (size_t)(n - t0) * hstride;
                CKL(launch_step(L.radius, kFwdHist, *tc, fp, c.st));
                float *t = cur; cur = prv; prv = t;
                const StepMaps *tt = tc; tc = tp; tp = tt;
            }
            g_prof.span(1, e0, g_prof.mark(c.st), nl);
        }
        nl = 0;
        e0 = g_prof.mark(c.st);
        // adjoint steps m = t1 .. t0+1, imaging with Lap(U^{m-1})
        for (int m = t1; m >= t0 + 1; --m) {
            ap.out = mprv;
            ap.step = m;
            ap.hist = hist + (size_t)(m - 1 - t0) * hstride;
            ap.hist_slot = m - 1 - t0;
            CKL(launch_step(L.radius, kAdjoint, *tmc, ap, c.st));
            float *t = mcur; mcur = mprv; mprv = t;
            const StepMaps *tt = tmc; tmc = tmp; tmp = tt;
        }
        g_prof.span(2, e0, g_prof.mark(c.st), nl);
    }
    // 4. (2/C) scaling, fold of the absorbing layer, FP64 reduction over transmits
    nl = 0;
    e0 = g_prof.mark(c.st);
    CKL(launch_fold(g_shot, sos, grad, c.at<double>(L.o_fold), L.n_maps, L.n_tx, L.Nx, L.Nz, L.P, L.slice, L.pitch,
                    c.st));
    ++nl;
    g_prof.span(3, e0, g_prof.mark(c.st), nl);
    return DUFWI_OK;
}

}  // extern "C"
