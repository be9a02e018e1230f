// C-ABI of the library (declared in include/nfmimo.h): context, geometry
// validation and upload, launch planning, SPGM driver, power iteration and
// FP64 objective.  Every step of the path runs in the kernels of this library;
// the host only validates, plans and enqueues.
#include "nfmimo.h"
#include "nfm_kernels.cuh"
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace nfm;

namespace {

thread_local std::string g_create_error;

// NVTX range around an entry point (tracing aid: a profiler shows the library's calls on its timeline;
// without one attached the push and pop cost a branch each)
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
};

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct FwdPlan {
    int VS, nt, n_groups, n_slots, n_chunks, base, rem;
    size_t smem;
    size_t partial_bytes;
};

}  // namespace

struct nfm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int num_sms = 0;
    size_t smem_optin = 0;

    bool has_geom = false;
    int T = 0, R = 0, K = 0, K1 = 0, P = 0;
    long long N = 0, M = 0;
    nfm_grid grid{};
    double c = 0, f0 = 0, df = 0;
    GridDesc gd{};
    PhaseConsts ph{};

    AntTile* d_ant = nullptr;
    double* d_ant_xyz = nullptr;
    bool points = false;          // explicit voxel positions (nfm_set_geometry_points)
    float4* d_pts = nullptr;      // points: per-voxel offsets from the tile centre [n_tiles * 128]
    double* d_tile_c = nullptr;   // points: tile centres [n_tiles][3]
    double* d_vox_xyz = nullptr;  // points: voxel positions [N][3]
    bool uniform = true;          // equally spaced frequencies (recurrence / tensor-core paths)
    float* d_antk = nullptr;      // general frequencies: [(T+R) * n_tiles * K] reduced phases
    float2* d_fkc = nullptr;      // general frequencies: f_k / c as hi + lo
    float2* d_pulse = nullptr;
    int* d_pairs_all = nullptr;
    int* d_err = nullptr;
    double* d_red = nullptr;   // [RED_BLOCKS] partials + 8 scalars

    void* d_partial = nullptr;
    size_t partial_cap = 0;
    void* d_resid = nullptr;
    size_t resid_cap = 0;
    void* d_v = nullptr;
    size_t v_cap = 0;
    void* d_g = nullptr;
    size_t g_cap = 0;
    void* d_y = nullptr;
    size_t y_cap = 0;
    void* d_hy = nullptr;
    size_t hy_cap = 0;
    void* d_hs = nullptr;
    size_t hs_cap = 0;
    void* d_hperm = nullptr;
    size_t hperm_cap = 0;
    void* d_prox_partial = nullptr;
    size_t prox_partial_cap = 0;
    void* d_bmat = nullptr;
    size_t bmat_cap = 0;
    void* d_bscale = nullptr;
    size_t bscale_cap = 0;
    int precision = NFM_FP32;
    int hooks = 0;                        // test hooks (nfm_set_test_hooks)
    unsigned long long tc_wait_ns = 1000000000ull;   // limit of one bounded wait on the tensor core
    double reg_w1 = 1.0, reg_w2 = 0.0;    // R(s) = w1 ||s||_1 + (w2/2) ||s||_2^2
    double reg_w3 = 0.0;                  //      + w3 sum over 2 x 2 x 1 voxel blocks of ||s_g||_2
    unsigned long long scratch_gen = 0;   // bumped whenever a scratch buffer is (re)allocated
    bool adj_tc_attr[2][MAX_K1 + 1] = {};

    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Pending { int kind, a, b; };
    std::vector<Pending> pending;

    int fwd_occ[MAX_K1 + 1] = {};
    bool fwd_attr[MAX_K1 + 1] = {};
    bool adj_attr[MAX_K1 + 1] = {};

    // Chebyshev expansion of the frequency dependence (equally spaced frequencies)
    int algorithm = NFM_ALGO_AUTO;
    float* d_cheb = nullptr;      // [cheb_kpad][cheb_L] b_l(k)
    int cheb_L = 0;               // 0: not available for this geometry
    int cheb_kpad = 0;
    float cheb_tau = 0.f;         // t = tau * delta
    double cheb_zmax = 0.0;       // largest |z_k| (the band edges)
    float cheb_fc_hi = 0.f, cheb_fc_lo = 0.f;   // band centre f_c / c, hi + lo
    bool fwd_cheb_attr[CHEB_MAX_L + 1][2] = {};
    bool adj_cheb_attr[CHEB_MAX_L + 1] = {};
    bool adj_cheb_tc_attr[2][CHEB_MAX_L + 1] = {};
    bool fwd_cheb_tc_attr[2][CHEB_MAX_L + 1] = {};
    // the FP32 expansion adjoint's blocks of two tiles along z (regular grids): their grid descriptor,
    // antenna-block table and expansion table (cheb_L2 = 0: not set up, the adjoint runs over the tiles)
    GridDesc gd2{};
    AntTile* d_ant2 = nullptr;
    float* d_cheb2 = nullptr;
    int cheb_L2 = 0;
    float cheb_tau2 = 0.f;
    bool adj_cheb2_attr[CHEB_MAX_L + 1] = {};
    bool fwd_cheb2_attr[CHEB_MAX_L + 1][2] = {};
    // launch shapes of the expansion forward chosen by nfm_autotune, per minibatch size
    struct FwdShape { int n_pairs, threads, group, pch, chunks; bool direct; };
    std::vector<FwdShape> fwd_tuned;
};

namespace {

int failv(nfm_ctx* ctx, int code, const char* fmt, va_list ap)
{
    char buf[512];
    vsnprintf(buf, sizeof(buf), fmt, ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_error = buf;
    return code;
}

int fail(nfm_ctx* ctx, int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    int r = failv(ctx, code, fmt, ap);
    va_end(ap);
    return r;
}

#define NFM_CK(call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(ctx, NFM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

#define NFM_TRY(expr)             \
    do {                          \
        int r_ = (expr);          \
        if (r_ != NFM_OK) return r_; \
    } while (0)

int ensure(nfm_ctx* ctx, void** p, size_t* cap, size_t bytes)
{
    if (*cap >= bytes && *p) return NFM_OK;
    if (*p) {
        cudaError_t e = cudaFree(*p);   // synchronises the device before release
        *p = nullptr;
        *cap = 0;
        if (e != cudaSuccess) return fail(ctx, NFM_ERR_CUDA, "cudaFree failed: %s", cudaGetErrorString(e));
    }
    size_t want = bytes < 256 ? 256 : bytes;
    ++ctx->scratch_gen;
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(ctx, NFM_ERR_NOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    *cap = want;
    return NFM_OK;
}

void free_ptr(void* p)
{
    if (p) cudaFree(p);
}

OpDesc op_desc(const nfm_ctx* ctx)
{
    OpDesc op;
    op.g = ctx->gd;
    op.ph = ctx->ph;
    op.ant = ctx->d_ant;
    op.pulse = ctx->d_pulse;
    op.T = ctx->T;
    op.R = ctx->R;
    op.K = ctx->K;
    op.K1 = ctx->K1;
    op.P = ctx->P;
    op.err = ctx->d_err;
    op.wait_ns = ctx->tc_wait_ns;
    op.hooks = ctx->hooks;
    // extents for the bounds-checked build; the test hook halves them so that a check trips on an access
    // that is in fact inside its buffer
    const long long shrink = (ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1;
    op.n_vox = ctx->N / shrink;
    op.m_rows = ctx->M / shrink;
    return op;
}

int require_geom(nfm_ctx* ctx)
{
    if (!ctx) return NFM_ERR_ARG;
    if (!ctx->has_geom) return fail(ctx, NFM_ERR_STATE, "no geometry: call nfm_set_geometry first");
    return NFM_OK;
}

int check_ptr(nfm_ctx* ctx, const void* p, const char* name, size_t align)
{
    if (!p) return fail(ctx, NFM_ERR_ARG, "%s is NULL", name);
    if (((uintptr_t)p) % align) return fail(ctx, NFM_ERR_ARG, "%s is not %zu-byte aligned", name, align);
    return NFM_OK;
}

// Record a timing event on the context stream when profiling is on; returns
// its pool index or -1.
int prof_mark(nfm_ctx* ctx)
{
    if (!ctx->prof) return -1;
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return -1;
        ctx->ev_pool.push_back(ev);
    }
    int i = (int)ctx->ev_used++;
    if (cudaEventRecord(ctx->ev_pool[i], ctx->stream) != cudaSuccess) return -1;
    return i;
}

void prof_pair(nfm_ctx* ctx, int kind, int a, int b)
{
    if (ctx->prof && a >= 0 && b >= 0) ctx->pending.push_back({kind, a, b});
}

// b_l(k), l < L, of exp(-j z t) = sum_l (-j)^l b_l T_l(t) at z = k z_step (b_0 = J_0(z),
// b_l = 2 J_l(z)), by Chebyshev-Gauss quadrature of (eps_l / pi) int_0^pi e^{-j z cos th} cos(l th) dth
// with Q = 2L + 64 nodes (exact up to aliasing from degree >= 2Q - L).  FP64, row-major [K][L].
// Multiplier of the division n / d = umulhi(n, m) = floor(n m / 2^32) for 0 <= n < n_max: m = floor(2^32/d) + 1
// = 2^32/d + e with 0 < e <= 1, so n m / 2^32 = n/d + n e / 2^32, and the added n e / 2^32 < 1/d keeps the
// floor exact while n_max d <= 2^32 (Granlund and Montgomery, division by invariant integers using
// multiplication).  0 (plain division) when that bound fails or d = 1 (m would not fit 32 bits).
unsigned tile_div_magic(long long n_max, int d)
{
    if (d < 2 || n_max * (long long)d > (1ll << 32)) return 0u;
    return (unsigned)((1ull << 32) / (unsigned long long)d + 1ull);
}

// Truncation budget of the expansion: the dropped terms' coefficients at the band edge, sum_{l >= L}
// |b_l(z_max)|, bound the relative error of every element (|T_l(t)| <= 1); 2e-6 keeps it a fifth of the
// FP32 operator's 1e-5 relative bound and of the order of the FP32 rounding error, and well below it in
// the mean over the band (the tail falls fast as |z| drops from the edge).
constexpr double CHEB_TAIL = 2e-6;

void cheb_coefficients(double z_step, double k_center, int K, int L, double* out)
{
    const double pi = 3.14159265358979323846;
    const int Q = 2 * L + 64;
    std::vector<double> cth(Q), th(Q);
    for (int q = 0; q < Q; ++q) {
        th[q] = pi * (q + 0.5) / Q;
        cth[q] = std::cos(th[q]);
    }
    for (int k = 0; k < K; ++k) {
        const double z = (k - k_center) * z_step;
        for (int l = 0; l < L; ++l) {
            double re = 0.0, im = 0.0;
            for (int q = 0; q < Q; ++q) {
                const double w = std::cos(l * th[q]);
                re += std::cos(z * cth[q]) * w;
                im -= std::sin(z * cth[q]) * w;
            }
            const double eps = l == 0 ? 1.0 : 2.0;
            re *= eps / Q;
            im *= eps / Q;
            // a_l = (-j)^l b_l  =>  b_l = Re(j^l a_l)
            double b;
            switch (l & 3) {
            case 0: b = re; break;
            case 1: b = -im; break;
            case 2: b = -re; break;
            default: b = im; break;
            }
            out[(size_t)k * L + l] = b;
        }
    }
}

// Chebyshev expansion set-up for equally spaced frequencies: the FP64 range of
// delta = D - D_c over every (pair, tile), the scale tau with |t| <= 0.95, the
// band centre k_c = (K - 1)/2 (the expansion covers e^{-j z_k t} with
// z_k = (k - k_c) z_step, |z_k| <= z_step (K - 1)/2), the number of terms L
// (even, tail below CHEB_TAIL at the band edges) and the table.
int setup_cheb(nfm_ctx* ctx, const GridDesc& gd, const AntSetup& as, int K, double f0, double df, double c)
{
    unsigned long long* d_mx = nullptr;
    unsigned long long bits = 0;
    cudaError_t e = cudaMalloc((void**)&d_mx, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_mx, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = launch_cheb_range(gd, as, d_mx, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d_mx, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
    free_ptr(d_mx);
    if (e != cudaSuccess) return fail(ctx, NFM_ERR_CUDA, "expansion range: %s", cudaGetErrorString(e));
    double dmax;
    memcpy(&dmax, &bits, sizeof(dmax));
    const double margin = 0.95;
    const double span = 2.0 * dmax;                 // |delta| = |d_T - d_cT + d_R - d_cR| <= span
    if (!(span > 0)) return NFM_OK;                 // degenerate: keep the direct path
    const double z_step = 2.0 * 3.14159265358979323846 * df * span / (c * margin);
    const double k_center = 0.5 * (K - 1);
    const double zmax = z_step * k_center;
    // tail of the expansion at the band edges (|z| = zmax; |b_l(-z)| = |b_l(z)|)
    const int LP = 80;
    std::vector<double> probe(2 * LP);
    cheb_coefficients(zmax, 0.0, 2, LP, probe.data());   // rows z = 0 and z = zmax
    int L = 0;
    for (int cand = CHEB_MIN_L; cand <= CHEB_MAX_L; cand += 2) {
        double tail = 0.0;
        for (int l = cand; l < LP; ++l) tail += std::fabs(probe[LP + l]);
        if (tail < CHEB_TAIL) {
            L = cand;
            break;
        }
    }
    if (L == 0) return NFM_OK;                      // too many terms: the direct path stays
    const int kpad = (K + 3) & ~3;
    const int ls = (L + 3) & ~3;                    // table row stride, zero beyond L
    std::vector<double> b((size_t)K * L);
    cheb_coefficients(z_step, k_center, K, L, b.data());
    std::vector<float> hb((size_t)kpad * ls, 0.f);
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < L; ++l) hb[(size_t)k * ls + l] = (float)b[(size_t)k * L + l];
    e = cudaMalloc((void**)&ctx->d_cheb, hb.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_cheb, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_ptr(ctx->d_cheb);
        ctx->d_cheb = nullptr;
        return fail(ctx, NFM_ERR_NOMEM, "expansion table: %s", cudaGetErrorString(e));
    }
    ctx->cheb_L = L;
    ctx->cheb_kpad = kpad;
    ctx->cheb_tau = (float)(margin / span);
    ctx->cheb_zmax = zmax;
    const double fcc = (f0 + k_center * df) / c;
    ctx->cheb_fc_hi = (float)fcc;
    ctx->cheb_fc_lo = (float)(fcc - (double)ctx->cheb_fc_hi);
    return NFM_OK;
}

// The FP32 expansion adjoint's blocks of two tiles along z (8 x 4 x 8 voxels, regular grids): a grid
// descriptor over the blocks, the FP64 antenna-block rows (centres given explicitly to ant_setup_kernel)
// and an expansion table for the larger span.  |d - d_c| <= |u| (triangle inequality), so the block's
// corner offset bounds delta.  Leaves cheb_L2 = 0 (the operator stays on the tiles) where the span needs
// more terms than the block kernels are built for, or where the grid has fewer blocks than the GPU has
// SMs (small grids keep twice the CTAs of the tiles).
int setup_blocks2(nfm_ctx* ctx, const nfm_grid& g, const GridDesc& gd, const AntSetup& as, int K, double df, double c)
{
    constexpr int TZ2 = 2 * TILE_Z;
    GridDesc g2 = gd;
    g2.tiles_z = (g.nz + TZ2 - 1) / TZ2;
    g2.n_tiles = g2.tiles_x * g2.tiles_y * g2.tiles_z;
    g2.mx = tile_div_magic(g2.n_tiles, g2.tiles_x);
    g2.my = tile_div_magic(g2.n_tiles, g2.tiles_y);
    if (g2.n_tiles < ctx->num_sms) return NFM_OK;
    const double hx = 0.5 * (TILE_X - 1) * g.dx, hy = 0.5 * (TILE_Y - 1) * g.dy, hz = 0.5 * (TZ2 - 1) * g.dz;
    const double span = 2.0 * std::sqrt(hx * hx + hy * hy + hz * hz);
    const double margin = 0.95;
    const double z_step = 2.0 * 3.14159265358979323846 * df * span / (c * margin);
    const double k_center = 0.5 * (K - 1);
    const int LP = 80;
    std::vector<double> probe(2 * LP);
    cheb_coefficients(z_step * k_center, 0.0, 2, LP, probe.data());   // rows z = 0 and the band edge
    int L = 0;
    for (int cand = CHEB_MIN_L; cand <= CHEB_MAX_L; cand += 2) {
        double tail = 0.0;
        for (int l = cand; l < LP; ++l) tail += std::fabs(probe[LP + l]);
        if (tail < CHEB_TAIL) {
            L = cand;
            break;
        }
    }
    if (L == 0 || !adj_cheb_kernel_ptr(L, TZ2)) return NFM_OK;
    const int kpad = ctx->cheb_kpad, ls = (L + 3) & ~3;
    std::vector<double> b((size_t)K * L);
    cheb_coefficients(z_step, k_center, K, L, b.data());
    std::vector<float> hb((size_t)kpad * ls, 0.f);
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < L; ++l) hb[(size_t)k * ls + l] = (float)b[(size_t)k * L + l];
    std::vector<double> hc((size_t)g2.n_tiles * 3);
    for (int t = 0; t < g2.n_tiles; ++t) {   // block order: x fastest, then y, then z (as tile_coords)
        const int bx = t % g2.tiles_x, by = (t / g2.tiles_x) % g2.tiles_y, bz = t / (g2.tiles_x * g2.tiles_y);
        hc[3 * (size_t)t] = g.x0 + (bx * TILE_X + 0.5 * (TILE_X - 1)) * g.dx;
        hc[3 * (size_t)t + 1] = g.y0 + (by * TILE_Y + 0.5 * (TILE_Y - 1)) * g.dy;
        hc[3 * (size_t)t + 2] = g.z0 + (bz * TZ2 + 0.5 * (TZ2 - 1)) * g.dz;
    }
    double* d_c = nullptr;
    cudaError_t e = cudaMalloc((void**)&ctx->d_ant2, (size_t)as.n_ant * g2.n_tiles * sizeof(AntTile));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_cheb2, hb.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_c, hc.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_cheb2, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_c, hc.data(), hc.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        AntSetup a2 = as;
        a2.tile_c = d_c;
        a2.out = ctx->d_ant2;
        e = launch_ant_setup(g2, a2, ctx->stream);
    }
    if (e == cudaSuccess) e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
    free_ptr(d_c);
    if (e != cudaSuccess) {
        free_ptr(ctx->d_ant2);
        free_ptr(ctx->d_cheb2);
        ctx->d_ant2 = nullptr;
        ctx->d_cheb2 = nullptr;
        return fail(ctx, NFM_ERR_NOMEM, "adjoint block tables: %s", cudaGetErrorString(e));
    }
    ctx->gd2 = g2;
    ctx->cheb_L2 = L;
    ctx->cheb_tau2 = (float)(margin / span);
    return NFM_OK;
}

// Whether the Chebyshev kernels run for this context (equally spaced frequencies).
int use_cheb(nfm_ctx* ctx, bool& on, int n_pairs = -1)
{
    on = false;
    if (!ctx->uniform || ctx->algorithm == NFM_ALGO_DIRECT) return NFM_OK;
    if (ctx->cheb_L == 0) {
        if (ctx->algorithm == NFM_ALGO_CHEBYSHEV)
            return fail(ctx, NFM_ERR_ARG, "the Chebyshev expansion needs more than %d terms here", CHEB_MAX_L);
        return NFM_OK;
    }
    if (ctx->algorithm == NFM_ALGO_AUTO && n_pairs > 0)      // the autotuner may have preferred the direct form
        for (const auto& t : ctx->fwd_tuned)
            if (t.n_pairs == n_pairs && t.direct) return NFM_OK;
    on = true;
    return NFM_OK;
}

// max_chunks > 0 caps the number of voxel-tile chunks (the allocation-free forward holds every
// chunk's partial sums in a fixed array); the tile split below is the same for every count
int plan_forward(nfm_ctx* ctx, int n_pairs, FwdPlan* pl, long long max_chunks = 0)
{
    const int K1 = ctx->K1;
    pl->VS = 32 / K1;            // voxel subsets per warp; one warp per pair
    pl->nt = 32 * FWD_PC;
    pl->smem = fwd_smem_bytes(K1, pl->nt);
    const void* fn = fwd_kernel_ptr(K1);
    if (!ctx->fwd_attr[K1]) {
        NFM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin));
        ctx->fwd_attr[K1] = true;
    }
    if (pl->smem > ctx->smem_optin) return fail(ctx, NFM_ERR_ARG, "forward tile needs %zu B shared memory", pl->smem);
    int& occ = ctx->fwd_occ[K1];
    if (occ == 0) {
        NFM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, pl->nt, pl->smem));
        if (occ < 1) occ = 1;
    }
    pl->n_groups = (n_pairs + FWD_PC - 1) / FWD_PC;
    pl->n_slots = pl->n_groups * FWD_PC;
    long long G = (long long)ctx->num_sms * occ;
    long long nch = (G + pl->n_groups - 1) / pl->n_groups;
    if (nch < 1) nch = 1;
    if (nch > ctx->gd.n_tiles) nch = ctx->gd.n_tiles;
    if (nch > 65535) nch = 65535;
    if (max_chunks > 0 && nch > max_chunks) nch = max_chunks;
    pl->n_chunks = (int)nch;
    pl->base = ctx->gd.n_tiles / pl->n_chunks;
    pl->rem = ctx->gd.n_tiles % pl->n_chunks;
    pl->partial_bytes = (size_t)pl->n_chunks * pl->n_slots * ctx->K * sizeof(float2);
    return NFM_OK;
}

// out[b*K + k] = (A_B s)[b, k] (- y_obs[pair_b*K + k] if y_obs; 0 where fmask[k] == 0)
void plan_forward_general(const nfm_ctx* ctx, int n_pairs, FwdPlan* plp)
{
    FwdPlan& pl = *plp;
    pl.n_groups = (n_pairs + FWD_PC - 1) / FWD_PC;
    pl.n_slots = pl.n_groups * FWD_PC;
    long long G = (long long)ctx->num_sms * 4;
    long long nch = (G + pl.n_groups - 1) / pl.n_groups;
    if (nch > ctx->gd.n_tiles) nch = ctx->gd.n_tiles;
    if (nch > 65535) nch = 65535;
    if (nch < 1) nch = 1;
    pl.n_chunks = (int)nch;
    pl.base = ctx->gd.n_tiles / pl.n_chunks;
    pl.rem = ctx->gd.n_tiles % pl.n_chunks;
    pl.partial_bytes = (size_t)pl.n_chunks * pl.n_slots * ctx->K * sizeof(float2);
}

int enqueue_forward_general(nfm_ctx* ctx, const int* pairs, int n_pairs, const float2* s, const float2* y_obs,
                            float2* out, const unsigned char* fmask)
{
    FwdPlan pl;
    plan_forward_general(ctx, n_pairs, &pl);
    NFM_TRY(ensure(ctx, &ctx->d_partial, &ctx->partial_cap, pl.partial_bytes));
    OpDesc op = op_desc(ctx);
    GenDesc gdsc{ctx->d_antk, ctx->d_fkc};
    FwdArgs a;
    a.pairs = pairs;
    a.n_pairs = n_pairs;
    a.s = s;
    a.partial = (float2*)ctx->d_partial;
    a.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    a.n_slots = pl.n_slots;
    a.VS = 1;
    a.tiles_base = pl.base;
    a.tiles_rem = pl.rem;
    const int e0 = prof_mark(ctx);
    NFM_CK(launch_fwd_general(op, gdsc, a, dim3(pl.n_groups, pl.n_chunks), ctx->stream));
    const int e1 = prof_mark(ctx);
    ReduceArgs ra;
    ra.partial = (const float2*)ctx->d_partial;
    ra.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    ra.n_chunks = pl.n_chunks;
    ra.n_slots = pl.n_slots;
    ra.n_out = n_pairs * ctx->K;
    ra.pairs = pairs;
    ra.y_obs = y_obs;
    ra.fmask = fmask;
    ra.out = out;
    NFM_CK(launch_fwd_reduce(op, ra, ctx->stream));
    const int e2 = prof_mark(ctx);
    prof_pair(ctx, 0, e0, e1);
    prof_pair(ctx, 1, e1, e2);
    return NFM_OK;
}

// Launch shape of the expansion forward: CTA size, pairs per CTA and tile chunks.
struct ChebShape {
    int threads, group, pch, n_groups, n_slots;
    long long nch;
    size_t smem;
    int occ;                 // resident CTAs per SM (0 when the chunk count was given)
    int tz = TILE_Z;         // z extent of the voxel blocks: TILE_Z (tiles) or 2 TILE_Z (the adjoint's blocks)
};

// Default shape (threads = 128, 4 lanes per (pair, tile), pairs per CTA = the power of two >=
// n_pairs in [4, 32], about `waves` CTAs per resident slot, at least one full stage of tiles per
// chunk), or the one given (`chunks` > 0: any count up to one tile per chunk; a chunk shorter than a
// stage leaves the stage's remaining slots idle).
int cheb_shape(nfm_ctx* ctx, int n_pairs, int threads, int group, int pch, double waves, long long chunks,
               ChebShape* sh, bool tiles_only = false)
{
    // on a regular grid the forward runs over the adjoint's blocks of two tiles along z (same tables)
    const bool blk = !tiles_only && ctx->cheb_L2 > 0 && !ctx->points &&
                     fwd_cheb_kernel_ptr(ctx->cheb_L2, group, 2 * TILE_Z) != nullptr;
    const int LT = blk ? ctx->cheb_L2 : ctx->cheb_L, KP = ctx->cheb_kpad;
    const int tz = blk ? 2 * TILE_Z : TILE_Z;
    const long long n_tiles = blk ? ctx->gd2.n_tiles : ctx->gd.n_tiles;
    const int ng = threads / group;
    if (pch <= 0) {
        pch = 4;
        while (pch < ng && pch < n_pairs) pch *= 2;
    }
    if (ctx->points && pch < ng / 2) pch = ng / 2;     // explicit positions: at most two tiles per stage
    if (ng % pch != 0) return fail(ctx, NFM_ERR_ARG, "pairs per CTA %d does not divide %d groups", pch, ng);
    const int TS = ng / pch;
    sh->threads = threads;
    sh->group = group;
    sh->pch = pch;
    sh->tz = tz;
    sh->smem = fwd_cheb_smem_bytes(LT, KP, pch, threads, group, ctx->points, tz);
    if (sh->smem > ctx->smem_optin) return fail(ctx, NFM_ERR_ARG, "expansion forward needs %zu B shared memory", sh->smem);
    const void* fn = fwd_cheb_kernel_ptr(LT, group, tz);
    if (!fn) return fail(ctx, NFM_ERR_ARG, "no expansion forward for L = %d, group %d", LT, group);
    bool& attr = blk ? ctx->fwd_cheb2_attr[LT][group == 8] : ctx->fwd_cheb_attr[LT][group == 8];
    if (!attr) {
        NFM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin));
        // all of the unified L1 / shared memory as shared memory: the CTA count per SM is set by shared memory
        NFM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        attr = true;
    }
    sh->n_groups = (n_pairs + pch - 1) / pch;
    sh->n_slots = sh->n_groups * pch;
    sh->occ = 0;                             // queried only for the default chunk count
    long long nch = chunks;
    if (nch <= 0) {
        int occ = 0;
        NFM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, sh->smem));
        if (occ < 1) occ = 1;
        sh->occ = occ;
        const long long G = (long long)(waves * ctx->num_sms * occ);
        nch = (G + sh->n_groups - 1) / sh->n_groups;
        const long long max_ch = (n_tiles + TS - 1) / TS;
        if (nch > max_ch) nch = max_ch;
    }
    if (nch > n_tiles) nch = n_tiles;
    if (nch > 65535) nch = 65535;
    if (nch < 1) nch = 1;
    sh->nch = nch;
    return NFM_OK;
}

int launch_cheb_forward_shape(nfm_ctx* ctx, const ChebShape& sh, const int* pairs, int n_pairs, const float2* s)
{
    const size_t partial_bytes = (size_t)sh.nch * sh.n_slots * ctx->K * sizeof(float2);
    NFM_TRY(ensure(ctx, &ctx->d_partial, &ctx->partial_cap, partial_bytes));
    const bool blk = sh.tz != TILE_Z;        // the adjoint's blocks and their tables
    ChebDesc cd{blk ? ctx->d_cheb2 : ctx->d_cheb, blk ? ctx->cheb_tau2 : ctx->cheb_tau,
                blk ? ctx->cheb_L2 : ctx->cheb_L, ctx->cheb_kpad, ctx->cheb_fc_hi, ctx->cheb_fc_lo};
    OpDesc op = op_desc(ctx);
    if (blk) {
        op.g = ctx->gd2;
        op.ant = ctx->d_ant2;
    }
    FwdArgs a;
    a.pairs = pairs;
    a.n_pairs = n_pairs;
    a.s = s;
    a.partial = (float2*)ctx->d_partial;
    a.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    a.n_slots = sh.n_slots;
    a.VS = sh.pch;
    a.tiles_base = (int)(op.g.n_tiles / sh.nch);
    a.tiles_rem = (int)(op.g.n_tiles % sh.nch);
    NFM_CK(launch_fwd_cheb(op, cd, a, dim3(sh.n_groups, (unsigned)sh.nch), sh.threads, sh.group, sh.tz, sh.smem,
                           ctx->stream));
    return NFM_OK;
}

// Tensor-core expansion forward (precision modes): 256-thread CTAs, 16, 32 or 64 pairs per CTA, one
// wave of two CTAs per SM over the voxel-tile chunks.
// launch shape of the tensor-core forward for n_pairs pairs: pairs per CTA, pair groups, voxel-tile chunks
void tc_fwd_shape(const nfm_ctx* ctx, int n_pairs, int* pch_out, int* groups_out, long long* nch_out)
{
    const int pch = n_pairs <= 16 ? 16 : n_pairs <= 32 ? 32 : 64;
    const int TS = 64 / pch;
    const int n_groups = (n_pairs + pch - 1) / pch;
    long long nch = (2LL * ctx->num_sms + n_groups - 1) / n_groups;
    const long long max_ch = (ctx->gd.n_tiles + TS - 1) / TS;
    if (nch > max_ch) nch = max_ch;
    if (nch > 65535) nch = 65535;
    if (nch < 1) nch = 1;
    *pch_out = pch;
    *groups_out = n_groups;
    *nch_out = nch;
}

int enqueue_forward_cheb_tc(nfm_ctx* ctx, const int* pairs, int n_pairs, const float2* s, const float2* y_obs,
                            float2* out, const unsigned char* fmask)
{
    const int LT = ctx->cheb_L;
    const bool f16 = ctx->precision == NFM_TC_FP16X3;
    int pch = 0, n_groups = 0;
    long long nch = 0;
    tc_fwd_shape(ctx, n_pairs, &pch, &n_groups, &nch);
    const size_t smem = fwd_cheb_tc_smem_bytes(LT, ctx->K, pch);
    if (smem > ctx->smem_optin) return fail(ctx, NFM_ERR_ARG, "tensor-core expansion forward needs %zu B shared memory", smem);
    if (!ctx->fwd_cheb_tc_attr[f16][LT]) {
        NFM_CK(cudaFuncSetAttribute(fwd_cheb_tc_kernel_ptr(LT, f16), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ctx->smem_optin));
        ctx->fwd_cheb_tc_attr[f16][LT] = true;
    }
    const int n_slots = n_groups * pch;
    NFM_TRY(ensure(ctx, &ctx->d_partial, &ctx->partial_cap, (size_t)nch * n_slots * ctx->K * sizeof(float2)));
    ChebDesc cd{ctx->d_cheb, ctx->cheb_tau, LT, ctx->cheb_kpad, ctx->cheb_fc_hi, ctx->cheb_fc_lo};
    FwdArgs a;
    a.pairs = pairs;
    a.n_pairs = n_pairs;
    a.s = s;
    a.partial = (float2*)ctx->d_partial;
    a.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    a.n_slots = n_slots;
    a.VS = pch;
    a.tiles_base = (int)(ctx->gd.n_tiles / nch);
    a.tiles_rem = (int)(ctx->gd.n_tiles % nch);
    OpDesc op = op_desc(ctx);
    const int e0 = prof_mark(ctx);
    NFM_CK(launch_fwd_cheb_tc(op, cd, a, dim3(n_groups, (unsigned)nch), f16, smem, ctx->stream));
    const int e1 = prof_mark(ctx);
    ReduceArgs ra;
    ra.partial = (const float2*)ctx->d_partial;
    ra.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    ra.n_chunks = (int)nch;
    ra.n_slots = n_slots;
    ra.n_out = n_pairs * ctx->K;
    ra.pairs = pairs;
    ra.y_obs = y_obs;
    ra.fmask = fmask;
    ra.out = out;
    NFM_CK(launch_fwd_reduce(op, ra, ctx->stream));
    const int e2 = prof_mark(ctx);
    prof_pair(ctx, 0, e0, e1);
    prof_pair(ctx, 1, e1, e2);
    return NFM_OK;
}

int enqueue_forward_cheb(nfm_ctx* ctx, const int* pairs, int n_pairs, const float2* s, const float2* y_obs,
                         float2* out, const unsigned char* fmask)
{
    if (ctx->precision != NFM_FP32) return enqueue_forward_cheb_tc(ctx, pairs, n_pairs, s, y_obs, out, fmask);
    ChebShape sh;
    bool tuned = false;
    for (const auto& t : ctx->fwd_tuned)
        if (t.n_pairs == n_pairs) {
            NFM_TRY(cheb_shape(ctx, n_pairs, t.threads, t.group, t.pch, 0.0, t.chunks, &sh));
            tuned = true;
            break;
        }
    if (!tuned) NFM_TRY(cheb_shape(ctx, n_pairs, CHEB_THREADS, CHEB_GROUP, 0, 2.0, 0, &sh));
    const int e0 = prof_mark(ctx);
    NFM_TRY(launch_cheb_forward_shape(ctx, sh, pairs, n_pairs, s));
    const int e1 = prof_mark(ctx);
    OpDesc op = op_desc(ctx);
    ReduceArgs ra;
    ra.partial = (const float2*)ctx->d_partial;
    ra.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    ra.n_chunks = (int)sh.nch;
    ra.n_slots = sh.n_slots;
    ra.n_out = n_pairs * ctx->K;
    ra.pairs = pairs;
    ra.y_obs = y_obs;
    ra.fmask = fmask;
    ra.out = out;
    NFM_CK(launch_fwd_reduce(op, ra, ctx->stream));
    const int e2 = prof_mark(ctx);
    prof_pair(ctx, 0, e0, e1);
    prof_pair(ctx, 1, e1, e2);
    return NFM_OK;
}

// Geometries with explicit voxel positions run the FP32 expansion kernels only.
int points_check(nfm_ctx* ctx, bool cheb)
{
    if (!ctx->points) return NFM_OK;
    if (!cheb) return fail(ctx, NFM_ERR_ARG, "explicit voxel positions need the Chebyshev-expansion operator");
    if (ctx->precision != NFM_FP32)
        return fail(ctx, NFM_ERR_ARG, "explicit voxel positions run the FP32 operator only (precision FP32)");
    return NFM_OK;
}

int enqueue_forward(nfm_ctx* ctx, const int* pairs, int n_pairs, const float2* s, const float2* y_obs,
                    float2* out, const unsigned char* fmask = nullptr)
{
    if (!ctx->uniform) return enqueue_forward_general(ctx, pairs, n_pairs, s, y_obs, out, fmask);
    bool cheb = false;
    NFM_TRY(use_cheb(ctx, cheb, n_pairs));
    NFM_TRY(points_check(ctx, cheb));
    if (cheb) return enqueue_forward_cheb(ctx, pairs, n_pairs, s, y_obs, out, fmask);
    FwdPlan pl;
    NFM_TRY(plan_forward(ctx, n_pairs, &pl));
    NFM_TRY(ensure(ctx, &ctx->d_partial, &ctx->partial_cap, pl.partial_bytes));
    OpDesc op = op_desc(ctx);
    FwdArgs a;
    a.pairs = pairs;
    a.n_pairs = n_pairs;
    a.s = s;
    a.partial = (float2*)ctx->d_partial;
    a.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    a.n_slots = pl.n_slots;
    a.VS = pl.VS;
    a.tiles_base = pl.base;
    a.tiles_rem = pl.rem;
    const int e0 = prof_mark(ctx);
    NFM_CK(launch_fwd_partial(op, a, dim3(pl.n_groups, pl.n_chunks), pl.nt, pl.smem, ctx->stream));
    const int e1 = prof_mark(ctx);
    ReduceArgs ra;
    ra.partial = (const float2*)ctx->d_partial;
    ra.partial_elems = (long long)(ctx->partial_cap / sizeof(float2)) / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    ra.n_chunks = pl.n_chunks;
    ra.n_slots = pl.n_slots;
    ra.n_out = n_pairs * ctx->K;
    ra.pairs = pairs;
    ra.y_obs = y_obs;
    ra.fmask = fmask;
    ra.out = out;
    NFM_CK(launch_fwd_reduce(op, ra, ctx->stream));
    const int e2 = prof_mark(ctx);
    prof_pair(ctx, 0, e0, e1);
    prof_pair(ctx, 1, e1, e2);
    return NFM_OK;
}

int enqueue_adjoint_tc(nfm_ctx* ctx, const int* pairs, int n_pairs, const float2* r, float2* g_out, float2* s,
                       float step, float alpha, float shrink)
{
    const int K1 = ctx->K1;
    const bool f16 = ctx->precision == NFM_TC_FP16X3;
    const size_t smem = adj_tc_smem_bytes(ADJ_TC_PCHUNK);
    if (!ctx->adj_tc_attr[f16][K1]) {
        NFM_CK(cudaFuncSetAttribute(adj_tc_kernel_ptr(K1, f16), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ctx->smem_optin));
        ctx->adj_tc_attr[f16][K1] = true;
    }
    NFM_TRY(ensure(ctx, &ctx->d_bmat, &ctx->bmat_cap, adj_tc_bmat_bytes(n_pairs)));
    NFM_TRY(ensure(ctx, &ctx->d_bscale, &ctx->bscale_cap, (size_t)n_pairs * sizeof(float)));
    AdjArgs a;
    a.pairs = pairs;
    a.n_pairs = n_pairs;
    a.r = r;
    a.r_elems = (long long)n_pairs * ctx->K / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    a.g_out = g_out;
    a.s = s;
    a.step = step;
    a.alpha = alpha;
    a.shrink = shrink;
    a.pchunk = ADJ_TC_PCHUNK;
    const int e0 = prof_mark(ctx);
    NFM_CK(launch_adjoint_tc(op_desc(ctx), a, f16, r, (unsigned char*)ctx->d_bmat, (float*)ctx->d_bscale, smem,
                             ctx->stream));
    prof_pair(ctx, 2, e0, prof_mark(ctx));
    return NFM_OK;
}

// alpha_g > 0: the fused update also shrinks 2 x 2 x 1 voxel blocks (expansion adjoints only)
int enqueue_adjoint(nfm_ctx* ctx, const int* pairs, int n_pairs, const float2* r, float2* g_out, float2* s,
                    float step, float alpha, float shrink = 1.0f, float alpha_g = 0.f)
{
    if (alpha_g > 0.f && s) {
        bool cheb = false;
        if (ctx->uniform) NFM_TRY(use_cheb(ctx, cheb, n_pairs));
        if (!cheb)
            return fail(ctx, NFM_ERR_ARG, "the group term of the regulariser needs the Chebyshev-expansion "
                                          "operator (equally spaced frequencies, algorithm auto or chebyshev)");
    }
    if (!ctx->uniform) {
        if (ctx->precision != NFM_FP32)
            return fail(ctx, NFM_ERR_ARG, "the tensor-core adjoint needs equally spaced frequencies");
        AdjArgs a;
        a.pairs = pairs;
        a.n_pairs = n_pairs;
        a.r = r;
        a.r_elems = (long long)n_pairs * ctx->K / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
        a.g_out = g_out;
        a.s = s;
        a.step = step;
        a.alpha = alpha;
        a.shrink = shrink;
        a.pchunk = GEN_ADJ_PCHUNK;
        GenDesc gdsc{ctx->d_antk, ctx->d_fkc};
        const int e0 = prof_mark(ctx);
        NFM_CK(launch_adj_general(op_desc(ctx), gdsc, a, ctx->stream));
        prof_pair(ctx, 2, e0, prof_mark(ctx));
        return NFM_OK;
    }
    bool cheb = false;
    NFM_TRY(use_cheb(ctx, cheb, n_pairs));
    NFM_TRY(points_check(ctx, cheb));
    if (ctx->points && alpha_g > 0.f && s)
        return fail(ctx, NFM_ERR_ARG, "the group term of the regulariser needs a regular voxel grid");
    if (ctx->precision != NFM_FP32) {
        if (!cheb) return enqueue_adjoint_tc(ctx, pairs, n_pairs, r, g_out, s, step, alpha, shrink);
        // expansion adjoint with its coefficient stage on the tensor cores
        const bool f16 = ctx->precision == NFM_TC_FP16X3;
        const int LT = ctx->cheb_L;
        const size_t smem = adj_cheb_tc_smem_bytes(ctx->K, LT);
        if (smem > ctx->smem_optin) return fail(ctx, NFM_ERR_ARG, "tensor-core expansion needs %zu B shared memory", smem);
        if (!ctx->adj_cheb_tc_attr[f16][LT]) {
            NFM_CK(cudaFuncSetAttribute(adj_cheb_tc_kernel_ptr(LT, f16), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ctx->smem_optin));
            // all of the unified L1 / shared memory as shared memory, so that two CTAs fit per SM
            NFM_CK(cudaFuncSetAttribute(adj_cheb_tc_kernel_ptr(LT, f16), cudaFuncAttributePreferredSharedMemoryCarveout,
                                        100));
            ctx->adj_cheb_tc_attr[f16][LT] = true;
        }
        AdjArgs a;
        a.pairs = pairs;
        a.n_pairs = n_pairs;
        a.r = r;
        a.r_elems = (long long)n_pairs * ctx->K / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    a.r_elems = (long long)n_pairs * ctx->K / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
        a.g_out = g_out;
        a.s = s;
        a.step = step;
        a.alpha = alpha;
        a.shrink = shrink;
        a.pchunk = 16;
        a.alpha_g = alpha_g;
        ChebDesc cd{ctx->d_cheb, ctx->cheb_tau, LT, ctx->cheb_kpad, ctx->cheb_fc_hi, ctx->cheb_fc_lo};
        const int e0 = prof_mark(ctx);
        NFM_CK(launch_adj_cheb_tc(op_desc(ctx), cd, a, f16, smem, ctx->stream));
        prof_pair(ctx, 2, e0, prof_mark(ctx));
        return NFM_OK;
    }
    if (cheb) {
        // on a regular grid the adjoint runs over blocks of two tiles along z (their own tables)
        const bool blk2 = ctx->cheb_L2 > 0 && !ctx->points;
        const int LT = blk2 ? ctx->cheb_L2 : ctx->cheb_L;
        const int tz = blk2 ? 2 * TILE_Z : TILE_Z;
        const size_t smem = adj_cheb_smem_bytes(LT, ctx->cheb_kpad, tz);
        const void* fn = adj_cheb_kernel_ptr(LT, tz);
        if (!fn) return fail(ctx, NFM_ERR_ARG, "no expansion adjoint for L = %d", LT);
        bool& attr = blk2 ? ctx->adj_cheb2_attr[LT] : ctx->adj_cheb_attr[LT];
        if (!attr) {
            NFM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin));
            // all of the unified L1 / shared memory as shared memory, so that eight (four) CTAs fit per SM
            NFM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            attr = true;
        }
        AdjArgs a;
        a.pairs = pairs;
        a.n_pairs = n_pairs;
        a.r = r;
        a.r_elems = (long long)n_pairs * ctx->K / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
        a.g_out = g_out;
        a.s = s;
        a.step = step;
        a.alpha = alpha;
        a.shrink = shrink;
        a.pchunk = adj_cheb_pchunk(tz);
        a.alpha_g = alpha_g;
        ChebDesc cd{blk2 ? ctx->d_cheb2 : ctx->d_cheb, blk2 ? ctx->cheb_tau2 : ctx->cheb_tau, LT, ctx->cheb_kpad,
                    ctx->cheb_fc_hi, ctx->cheb_fc_lo};
        OpDesc op = op_desc(ctx);
        if (blk2) {
            op.g = ctx->gd2;
            op.ant = ctx->d_ant2;
        }
        const int e0 = prof_mark(ctx);
        NFM_CK(launch_adj_cheb(op, cd, a, tz, smem, ctx->stream));
        prof_pair(ctx, 2, e0, prof_mark(ctx));
        return NFM_OK;
    }
    const int K1 = ctx->K1;
    size_t smem = adj_smem_bytes(K1, ADJ_PCHUNK);
    if (!ctx->adj_attr[K1]) {
        NFM_CK(cudaFuncSetAttribute(adj_kernel_ptr(K1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ctx->smem_optin));
        ctx->adj_attr[K1] = true;
    }
    AdjArgs a;
    a.pairs = pairs;
    a.n_pairs = n_pairs;
    a.r = r;
    a.r_elems = (long long)n_pairs * ctx->K / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    a.g_out = g_out;
    a.s = s;
    a.step = step;
    a.alpha = alpha;
    a.shrink = shrink;
    a.pchunk = ADJ_PCHUNK;
    const int e0 = prof_mark(ctx);
    NFM_CK(launch_adjoint(op_desc(ctx), a, smem, ctx->stream));
    prof_pair(ctx, 2, e0, prof_mark(ctx));
    return NFM_OK;
}

int check_flags(nfm_ctx* ctx)
{
    int flags = 0;
    NFM_CK(cudaMemcpy(&flags, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flags) {
        NFM_CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
        if (flags & ERRF_PAIR) return fail(ctx, NFM_ERR_ARG, "a pair index was outside [0, P)");
        if (flags & ERRF_TIMEOUT) return fail(ctx, NFM_ERR_TIMEOUT, "a bounded wait on the tensor core gave up");
        if (flags & ERRF_BOUNDS)
            return fail(ctx, NFM_ERR_STATE, "a kernel index fell outside its buffer (bounds-checked build)");
        return fail(ctx, NFM_ERR_NUMERIC, "device flag 0x%x", flags);
    }
    return NFM_OK;
}

int spgm_step_impl(nfm_ctx* ctx, const float2* y, float2* s, const int* pairs, int n_pairs, float eta,
                   float lambda)
{
    NFM_TRY(ensure(ctx, &ctx->d_resid, &ctx->resid_cap, (size_t)n_pairs * ctx->K * sizeof(float2)));
    float2* r = (float2*)ctx->d_resid;
    NFM_TRY(enqueue_forward(ctx, pairs, n_pairs, s, y, r));
    const double B = (double)n_pairs * ctx->K;
    NFM_TRY(enqueue_adjoint(ctx, pairs, n_pairs, r, nullptr, s, (float)(eta / B),
                            (float)((double)eta * lambda * ctx->reg_w1),
                            (float)(1.0 / (1.0 + (double)eta * lambda * ctx->reg_w2)),
                            (float)((double)eta * lambda * ctx->reg_w3)));
    return NFM_OK;
}

int spgm_epoch_impl(nfm_ctx* ctx, const float2* y, float2* s, const int* perm, int bp, float eta, float lambda)
{
    NFM_TRY(ensure(ctx, &ctx->d_resid, &ctx->resid_cap, (size_t)bp * ctx->K * sizeof(float2)));
    for (int c0 = 0; c0 < ctx->P; c0 += bp) {
        int nb = ctx->P - c0 < bp ? ctx->P - c0 : bp;
        NFM_TRY(spgm_step_impl(ctx, y, s, perm + c0, nb, eta, lambda));
    }
    return NFM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int nfm_create(nfm_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(nullptr, NFM_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, NFM_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, NFM_ERR_ARG, "device %d out of range (%d)", device, ndev);
    DevGuard guard(device);
    nfm_ctx* ctx = new nfm_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    int v = 0;
    if ((e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess) {
        delete ctx;
        return fail(nullptr, NFM_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    }
    ctx->smem_optin = (size_t)v;
    if ((e = cudaMalloc((void**)&ctx->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_red, (RED_BLOCKS + 8) * sizeof(double))) != cudaSuccess ||
        (e = cudaMemset(ctx->d_err, 0, sizeof(int))) != cudaSuccess) {
        free_ptr(ctx->d_err);
        free_ptr(ctx->d_red);
        delete ctx;
        return fail(nullptr, NFM_ERR_NOMEM, "context allocation: %s", cudaGetErrorString(e));
    }
    *out = ctx;
    return NFM_OK;
}

void nfm_destroy(nfm_ctx* ctx)
{
    if (!ctx) return;
    DevGuard guard(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    void* ps[] = {ctx->d_ant, ctx->d_ant_xyz, ctx->d_pulse, ctx->d_antk, ctx->d_fkc, ctx->d_pairs_all, ctx->d_err, ctx->d_red,
                  ctx->d_partial, ctx->d_resid, ctx->d_v, ctx->d_g, ctx->d_y, ctx->d_hy, ctx->d_hs, ctx->d_hperm,
                  ctx->d_prox_partial, ctx->d_bmat, ctx->d_bscale, ctx->d_cheb, ctx->d_ant2, ctx->d_cheb2,
                  ctx->d_pts, ctx->d_tile_c,
                  ctx->d_vox_xyz};
    for (void* p : ps) free_ptr(p);
    for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
    delete ctx;
}

const char* nfm_last_error(const nfm_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int nfm_set_stream(nfm_ctx* ctx, void* cuda_stream)
{
    if (!ctx) return NFM_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return NFM_OK;
}

}  // extern "C"

namespace {
// Geometry set-up shared by the regular grid (grid != NULL) and explicit voxel positions (vox_xyz [n_vox][3],
// host FP64; voxel n in slot n % 128 of tile n / 128).
int set_geometry_impl(nfm_ctx* ctx, const double* tx_xyz, int T, const double* rx_xyz, int R, const double* freq_hz,
                      int K, const double* pulse_re_im, const nfm_grid* grid, const double* vox_xyz, long long n_vox,
                      double c)
{
    if (!ctx) return NFM_ERR_ARG;
    DevGuard guard(ctx->device);
    const bool pts = grid == nullptr;
    if (!tx_xyz || !rx_xyz || !freq_hz || (!grid && !vox_xyz)) return fail(ctx, NFM_ERR_ARG, "NULL geometry array");
    if (T < 1 || R < 1) return fail(ctx, NFM_ERR_ARG, "need T >= 1 and R >= 1 (got %d, %d)", T, R);
    if (K < 1 || K > K2 * MAX_K1) return fail(ctx, NFM_ERR_ARG, "K = %d outside [1, %d]", K, K2 * MAX_K1);
    if ((long long)T * R > (1LL << 30)) return fail(ctx, NFM_ERR_ARG, "too many pairs");
    nfm_grid g{};
    long long N = 0;
    if (pts) {
        if (n_vox < 1 || n_vox >= (1LL << 31) - TILE_V)
            return fail(ctx, NFM_ERR_ARG, "N = %lld voxels outside [1, 2^31 - 129]", n_vox);
        for (long long i = 0; i < 3 * n_vox; ++i)
            if (!std::isfinite(vox_xyz[i])) return fail(ctx, NFM_ERR_ARG, "non-finite voxel coordinate");
        N = n_vox;
        g.nx = (int)N;
        g.ny = g.nz = 1;
    } else {
        g = *grid;
        if (g.nx < 1 || g.ny < 1 || g.nz < 1) return fail(ctx, NFM_ERR_ARG, "grid dimensions must be >= 1");
        N = (long long)g.nx * g.ny * g.nz;
        if (N >= (1LL << 31)) return fail(ctx, NFM_ERR_ARG, "N = %lld voxels exceeds 2^31 - 1", N);
        const double gv[6] = {g.x0, g.y0, g.z0, g.dx, g.dy, g.dz};
        for (double x : gv)
            if (!std::isfinite(x)) return fail(ctx, NFM_ERR_ARG, "non-finite grid parameter");
        if (!(g.dx > 0 && g.dy > 0 && g.dz > 0)) return fail(ctx, NFM_ERR_ARG, "grid steps must be > 0");
    }
    if (!(c > 0) || !std::isfinite(c)) return fail(ctx, NFM_ERR_ARG, "c must be finite and > 0");
    for (int i = 0; i < 3 * T; ++i)
        if (!std::isfinite(tx_xyz[i])) return fail(ctx, NFM_ERR_ARG, "non-finite TX coordinate");
    for (int i = 0; i < 3 * R; ++i)
        if (!std::isfinite(rx_xyz[i])) return fail(ctx, NFM_ERR_ARG, "non-finite RX coordinate");
    for (int k = 0; k < K; ++k)
        if (!std::isfinite(freq_hz[k]) || !(freq_hz[k] > 0)) return fail(ctx, NFM_ERR_ARG, "frequency %d invalid", k);
    if (pulse_re_im)
        for (int k = 0; k < 2 * K; ++k)
            if (!std::isfinite(pulse_re_im[k])) return fail(ctx, NFM_ERR_ARG, "non-finite pulse spectrum");
    const double f0 = freq_hz[0];
    const double df = K > 1 ? (freq_hz[K - 1] - freq_hz[0]) / (K - 1) : 0.0;
    bool uniform = true;
    for (int k = 0; k < K; ++k) {
        double want = f0 + k * df;
        if (std::fabs(freq_hz[k] - want) > 1e-9 * std::fabs(freq_hz[K - 1])) uniform = false;
    }
    if (pts && !uniform)
        return fail(ctx, NFM_ERR_ARG, "explicit voxel positions need equally spaced frequencies");
    if (pts) {                               // every antenna at least 1e-6 m from every voxel
        for (int a = 0; a < T + R; ++a) {
            const double* p = a < T ? tx_xyz + 3 * a : rx_xyz + 3 * (a - T);
            for (long long n = 0; n < N; ++n) {
                const double* v = vox_xyz + 3 * n;
                const double d2 = (p[0] - v[0]) * (p[0] - v[0]) + (p[1] - v[1]) * (p[1] - v[1]) +
                                  (p[2] - v[2]) * (p[2] - v[2]);
                if (d2 < 1e-12) return fail(ctx, NFM_ERR_ARG, "antenna %d lies within 1e-6 m of voxel %lld", a, n);
            }
        }
    }
    // smallest antenna-voxel distance (distance to the grid's bounding box)
    const double lo[3] = {g.x0, g.y0, g.z0};
    const double hi[3] = {g.x0 + (g.nx - 1) * g.dx, g.y0 + (g.ny - 1) * g.dy, g.z0 + (g.nz - 1) * g.dz};
    for (int a = 0; a < T + R && !pts; ++a) {
        const double* p = a < T ? tx_xyz + 3 * a : rx_xyz + 3 * (a - T);
        bool inside = true;
        double d2 = 0;
        for (int j = 0; j < 3; ++j) {
            double q = p[j] < lo[j] ? lo[j] : (p[j] > hi[j] ? hi[j] : p[j]);
            d2 += (p[j] - q) * (p[j] - q);
            if (p[j] < lo[j] || p[j] > hi[j]) inside = false;
        }
        if (inside || d2 < 1e-12)
            return fail(ctx, NFM_ERR_ARG, "antenna %d lies within 1e-6 m of the voxel grid", a);
    }

    // release the previous geometry
    free_ptr(ctx->d_ant);
    free_ptr(ctx->d_ant_xyz);
    free_ptr(ctx->d_pulse);
    free_ptr(ctx->d_pairs_all);
    free_ptr(ctx->d_antk);
    free_ptr(ctx->d_fkc);
    free_ptr(ctx->d_cheb);
    ctx->d_cheb = nullptr;
    ctx->cheb_L = 0;
    free_ptr(ctx->d_ant2);
    free_ptr(ctx->d_cheb2);
    ctx->d_ant2 = nullptr;
    ctx->d_cheb2 = nullptr;
    ctx->cheb_L2 = 0;
    ctx->fwd_tuned.clear();
    ctx->d_antk = nullptr;
    ctx->d_fkc = nullptr;
    ctx->d_ant = nullptr;
    ctx->d_ant_xyz = nullptr;
    ctx->d_pulse = nullptr;
    ctx->d_pairs_all = nullptr;
    free_ptr(ctx->d_pts);
    free_ptr(ctx->d_tile_c);
    free_ptr(ctx->d_vox_xyz);
    ctx->d_pts = nullptr;
    ctx->d_tile_c = nullptr;
    ctx->d_vox_xyz = nullptr;
    ctx->points = false;
    ctx->has_geom = false;

    GridDesc gd;
    gd.nx = g.nx;
    gd.ny = g.ny;
    gd.nz = g.nz;
    if (pts) {                               // tiles of 128 consecutive voxels
        gd.tiles_x = (int)((N + TILE_V - 1) / TILE_V);
        gd.tiles_y = gd.tiles_z = 1;
    } else {
        gd.tiles_x = (g.nx + TILE_X - 1) / TILE_X;
        gd.tiles_y = (g.ny + TILE_Y - 1) / TILE_Y;
        gd.tiles_z = (g.nz + TILE_Z - 1) / TILE_Z;
    }
    gd.n_tiles = gd.tiles_x * gd.tiles_y * gd.tiles_z;
    gd.mx = tile_div_magic(gd.n_tiles, gd.tiles_x);
    gd.my = tile_div_magic(gd.n_tiles, gd.tiles_y);
    auto split = [](double x, float& h, float& l) {
        h = (float)x;
        l = (float)(x - (double)h);
    };
    split(g.dx, gd.dx_hi, gd.dx_lo);
    split(g.dy, gd.dy_hi, gd.dy_lo);
    split(g.dz, gd.dz_hi, gd.dz_lo);
    PhaseConsts ph;
    split(f0 / c, ph.f0c_hi, ph.f0c_lo);
    ph.dfc = (float)(df / c);
    ph.dfc2 = (float)(K2 * df / c);

    const int n_ant = T + R;
    const int P = T * R;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&ctx->d_ant, (size_t)n_ant * gd.n_tiles * sizeof(AntTile))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_ant_xyz, (size_t)n_ant * 3 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_pairs_all, (size_t)P * sizeof(int))) != cudaSuccess)
        return fail(ctx, NFM_ERR_NOMEM, "geometry allocation: %s", cudaGetErrorString(e));
    double* hxyz = new double[3 * n_ant];
    memcpy(hxyz, tx_xyz, 3 * T * sizeof(double));
    memcpy(hxyz + 3 * T, rx_xyz, 3 * R * sizeof(double));
    int* hp = new int[P];
    for (int i = 0; i < P; ++i) hp[i] = i;
    e = cudaMemcpy(ctx->d_ant_xyz, hxyz, 3 * n_ant * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_pairs_all, hp, P * sizeof(int), cudaMemcpyHostToDevice);
    delete[] hxyz;
    delete[] hp;
    NFM_CK(e);
    if (pulse_re_im) {
        float* hpl = new float[2 * K];
        for (int i = 0; i < 2 * K; ++i) hpl[i] = (float)pulse_re_im[i];
        e = cudaMalloc((void**)&ctx->d_pulse, K * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemcpy(ctx->d_pulse, hpl, K * sizeof(float2), cudaMemcpyHostToDevice);
        delete[] hpl;
        NFM_CK(e);
    }
    AntSetup as;
    as.ant_xyz = ctx->d_ant_xyz;
    as.n_ant = n_ant;
    as.x0 = g.x0;
    as.y0 = g.y0;
    as.z0 = g.z0;
    as.dx = g.dx;
    as.dy = g.dy;
    as.dz = g.dz;
    as.f0c = f0 / c;
    as.dfc = df / c;
    as.dfc2 = K2 * df / c;
    as.out = ctx->d_ant;
    if (pts) {
        // per tile: the centre of its voxels' bounding box (FP64) and every voxel's offset from it (FP32,
        // with |u|^2 from the FP64 offset); slots past N stay at the centre
        const long long nt = gd.n_tiles;
        std::vector<double> hc((size_t)nt * 3);
        std::vector<float4> hu((size_t)nt * TILE_V, make_float4(0.f, 0.f, 0.f, 0.f));
        for (long long t = 0; t < nt; ++t) {
            const long long n0 = t * TILE_V, n1 = std::min(N, n0 + TILE_V);
            for (int j = 0; j < 3; ++j) {
                double mn = vox_xyz[3 * n0 + j], mx = mn;
                for (long long n = n0; n < n1; ++n) {
                    mn = std::min(mn, vox_xyz[3 * n + j]);
                    mx = std::max(mx, vox_xyz[3 * n + j]);
                }
                hc[3 * t + j] = 0.5 * (mn + mx);
            }
            for (long long n = n0; n < n1; ++n) {
                const double ux = vox_xyz[3 * n] - hc[3 * t], uy = vox_xyz[3 * n + 1] - hc[3 * t + 1],
                             uz = vox_xyz[3 * n + 2] - hc[3 * t + 2];
                hu[n] = make_float4((float)ux, (float)uy, (float)uz, (float)(ux * ux + uy * uy + uz * uz));
            }
        }
        e = cudaMalloc((void**)&ctx->d_pts, hu.size() * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_tile_c, hc.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_vox_xyz, (size_t)N * 3 * sizeof(double));
        if (e != cudaSuccess) return fail(ctx, NFM_ERR_NOMEM, "voxel position tables: %s", cudaGetErrorString(e));
        e = cudaMemcpy(ctx->d_pts, hu.data(), hu.size() * sizeof(float4), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(ctx->d_tile_c, hc.data(), hc.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->d_vox_xyz, vox_xyz, (size_t)N * 3 * sizeof(double), cudaMemcpyHostToDevice);
        NFM_CK(e);
        gd.pts = ctx->d_pts;
        as.tile_c = ctx->d_tile_c;
        as.vox_xyz = ctx->d_vox_xyz;
        as.n_vox = N;
        ctx->points = true;
    }
    NFM_CK(launch_ant_setup(gd, as, ctx->stream));
    if (!uniform) {
        // general frequencies: FP64 reduced phases per (antenna, tile, k) and f_k / c split hi + lo
        double* hfk = new double[K];
        float* hfkc = new float[2 * K];
        for (int k = 0; k < K; ++k) {
            hfk[k] = freq_hz[k] / c;
            hfkc[2 * k] = (float)hfk[k];
            hfkc[2 * k + 1] = (float)(hfk[k] - (double)hfkc[2 * k]);
        }
        double* d_fk = nullptr;
        e = cudaMalloc((void**)&ctx->d_antk, (size_t)n_ant * gd.n_tiles * K * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_fkc, (size_t)K * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc((void**)&d_fk, (size_t)K * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(d_fk, hfk, K * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(ctx->d_fkc, hfkc, K * sizeof(float2), cudaMemcpyHostToDevice);
        delete[] hfk;
        delete[] hfkc;
        if (e == cudaSuccess) e = launch_antk_setup(gd, as, d_fk, K, ctx->d_antk, ctx->stream);
        if (e == cudaSuccess) e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
        free_ptr(d_fk);
        if (e != cudaSuccess) return fail(ctx, NFM_ERR_CUDA, "general-frequency tables: %s", cudaGetErrorString(e));
    }
    if (uniform) NFM_TRY(setup_cheb(ctx, gd, as, K, f0, df, c));
    if (uniform && !pts && ctx->cheb_L > 0) NFM_TRY(setup_blocks2(ctx, g, gd, as, K, df, c));
    NFM_CK(ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize());
    if (pts && ctx->cheb_L == 0)
        return fail(ctx, NFM_ERR_ARG, "explicit voxel positions: the path-length spread of a run of 128 voxels needs "
                                      "more than %d expansion terms; order the voxels so that each run of 128 is compact",
                    CHEB_MAX_L);

    ctx->T = T;
    ctx->R = R;
    ctx->K = K;
    ctx->K1 = (K + K2 - 1) / K2;
    ctx->P = P;
    ctx->N = N;
    ctx->M = (long long)P * K;
    ctx->grid = g;
    ctx->c = c;
    ctx->f0 = f0;
    ctx->df = df;
    ctx->gd = gd;
    ctx->ph = ph;
    ctx->uniform = uniform;
    ctx->has_geom = true;
    return NFM_OK;
}
}  // namespace

extern "C" {

int nfm_set_geometry(nfm_ctx* ctx, const double* tx_xyz, int T, const double* rx_xyz, int R,
                     const double* freq_hz, int K, const double* pulse_re_im, const nfm_grid* grid, double c)
{
    TraceRange trace_("nfm_set_geometry");
    if (!grid) return ctx ? fail(ctx, NFM_ERR_ARG, "NULL grid") : NFM_ERR_ARG;
    return set_geometry_impl(ctx, tx_xyz, T, rx_xyz, R, freq_hz, K, pulse_re_im, grid, nullptr, 0, c);
}

int nfm_set_geometry_points(nfm_ctx* ctx, const double* tx_xyz, int T, const double* rx_xyz, int R,
                            const double* freq_hz, int K, const double* pulse_re_im, const double* vox_xyz,
                            long long n_vox, double c)
{
    TraceRange trace_("nfm_set_geometry_points");
    if (!vox_xyz) return ctx ? fail(ctx, NFM_ERR_ARG, "NULL voxel positions") : NFM_ERR_ARG;
    return set_geometry_impl(ctx, tx_xyz, T, rx_xyz, R, freq_hz, K, pulse_re_im, nullptr, vox_xyz, n_vox, c);
}

int nfm_set_regularizer(nfm_ctx* ctx, double w1, double w2)
{
    if (!ctx) return NFM_ERR_ARG;
    if (!(w1 >= 0) || !(w2 >= 0) || !std::isfinite(w1) || !std::isfinite(w2) || (w1 == 0 && w2 == 0))
        return fail(ctx, NFM_ERR_ARG, "regularizer weights must be finite, >= 0 and not both 0");
    ctx->reg_w1 = w1;
    ctx->reg_w2 = w2;
    return NFM_OK;
}

int nfm_set_group_weight(nfm_ctx* ctx, double w3)
{
    if (!ctx) return NFM_ERR_ARG;
    if (!(w3 >= 0) || !std::isfinite(w3)) return fail(ctx, NFM_ERR_ARG, "group weight must be finite and >= 0");
    ctx->reg_w3 = w3;
    return NFM_OK;
}

int nfm_set_precision(nfm_ctx* ctx, int mode)
{
    if (!ctx) return NFM_ERR_ARG;
    if (mode != NFM_FP32 && mode != NFM_TC_BF16X3 && mode != NFM_TC_FP16X3)
        return fail(ctx, NFM_ERR_ARG, "unknown precision mode %d", mode);
    ctx->precision = mode;
    return NFM_OK;
}

int nfm_set_algorithm(nfm_ctx* ctx, int algo)
{
    if (!ctx) return NFM_ERR_ARG;
    if (algo != NFM_ALGO_AUTO && algo != NFM_ALGO_DIRECT && algo != NFM_ALGO_CHEBYSHEV)
        return fail(ctx, NFM_ERR_ARG, "unknown algorithm %d", algo);
    ctx->algorithm = algo;
    return NFM_OK;
}

int nfm_algorithm_info(nfm_ctx* ctx, int* algo_in_use, int* n_terms, double* z_max)
{
    NFM_TRY(require_geom(ctx));
    bool cheb = false;
    NFM_TRY(use_cheb(ctx, cheb));
    if (algo_in_use) *algo_in_use = cheb ? NFM_ALGO_CHEBYSHEV : NFM_ALGO_DIRECT;
    if (n_terms) *n_terms = ctx->cheb_L;
    if (z_max) *z_max = ctx->cheb_zmax;
    return NFM_OK;
}

int nfm_expansion_info(nfm_ctx* ctx, int* n_terms, int* block_voxels)
{
    NFM_TRY(require_geom(ctx));
    const bool blk2 = ctx->cheb_L2 > 0 && !ctx->points;
    if (n_terms) *n_terms = blk2 ? ctx->cheb_L2 : ctx->cheb_L;
    if (block_voxels) *block_voxels = blk2 ? TILE_X * TILE_Y * 2 * TILE_Z : TILE_V;
    return NFM_OK;
}

int nfm_autotune(nfm_ctx* ctx, int n_pairs, int* algorithm_out, int* threads_out, int* group_out,
                 int* pairs_per_cta_out, int* chunks_out)
{
    TraceRange trace_("nfm_autotune");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1 || n_pairs > ctx->P) return fail(ctx, NFM_ERR_ARG, "n_pairs = %d outside [1, P]", n_pairs);
    bool cheb = false;
    NFM_TRY(use_cheb(ctx, cheb));
    if (!cheb) return fail(ctx, NFM_ERR_STATE, "the autotuner covers the expansion forward only");
    auto drop_entry = [&]() {
        for (size_t i = 0; i < ctx->fwd_tuned.size(); ++i)
            if (ctx->fwd_tuned[i].n_pairs == n_pairs) {
                ctx->fwd_tuned.erase(ctx->fwd_tuned.begin() + i);
                return;
            }
    };
    drop_entry();
    NFM_TRY(ensure(ctx, &ctx->d_v, &ctx->v_cap, (size_t)ctx->N * sizeof(float2)));
    NFM_TRY(ensure(ctx, &ctx->d_resid, &ctx->resid_cap, (size_t)n_pairs * ctx->K * sizeof(float2)));
    NFM_TRY(ensure(ctx, &ctx->d_g, &ctx->g_cap, (size_t)ctx->N * sizeof(float2)));
    NFM_CK(cudaMemsetAsync(ctx->d_v, 0, (size_t)ctx->N * sizeof(float2), ctx->stream));
    const bool prof = ctx->prof;
    const int algorithm = ctx->algorithm;
    ctx->prof = false;
    cudaEvent_t e0, e1;
    NFM_CK(cudaEventCreate(&e0));
    NFM_CK(cudaEventCreate(&e1));
    // Steps as SPGM runs them (forward + residual reduction + adjoint, dependent launches overlapping
    // through PDL): one warm-up and `reps` timed repetitions.
    auto time_step = [&](float& ms, int reps) -> int {
        for (int r = 0; r <= reps; ++r) {
            if (r == 1 && cudaEventRecord(e0, ctx->stream) != cudaSuccess)
                return fail(ctx, NFM_ERR_CUDA, "autotuner event failed");
            int q = enqueue_forward(ctx, ctx->d_pairs_all, n_pairs, (const float2*)ctx->d_v, nullptr,
                                    (float2*)ctx->d_resid);
            if (q == NFM_OK)
                q = enqueue_adjoint(ctx, ctx->d_pairs_all, n_pairs, (const float2*)ctx->d_resid, (float2*)ctx->d_g,
                                    nullptr, 0.f, 0.f);
            if (q != NFM_OK) return q;
        }
        if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return fail(ctx, NFM_ERR_CUDA, "autotuner timing failed");
        return NFM_OK;
    };
    float best = 1e30f;
    ChebShape best_sh{};
    std::vector<std::pair<float, ChebShape>> timed;
    const double waves[3] = {1.0, 2.0, 4.0};
    int rc = NFM_OK;
    ctx->algorithm = NFM_ALGO_CHEBYSHEV;
    for (int group : {4, 8}) {
        for (int threads : {64, 128}) {
            const int ng = threads / group;
            for (int pch = 4; pch <= ng && rc == NFM_OK; pch *= 2) {
                if (pch / 2 >= n_pairs && pch > 4) break;        // all groups beyond the pairs would idle
                // waves of whole-stage chunks, then one wave of (occ - 1) or occ CTAs on every SM with
                // chunks that may be shorter than a stage (even work per SM when stages are coarse)
                for (int cand = 0; cand < 5 && rc == NFM_OK; ++cand) {
                    ChebShape sh;
                    if (cand < 3) {
                        rc = cheb_shape(ctx, n_pairs, threads, group, pch, waves[cand], 0, &sh);
                    } else {
                        rc = cheb_shape(ctx, n_pairs, threads, group, pch, 1.0, 0, &sh);
                        const long long per_sm = sh.occ - (cand == 3 ? 1 : 0);
                        const long long want = (per_sm * ctx->num_sms + sh.n_groups - 1) / sh.n_groups;
                        if (rc != NFM_OK || per_sm < 1 || want <= sh.nch) continue;   // covered above
                        rc = cheb_shape(ctx, n_pairs, threads, group, pch, 0.0, want, &sh);
                    }
                    if (rc != NFM_OK) break;
                    drop_entry();
                    ctx->fwd_tuned.push_back({n_pairs, sh.threads, sh.group, sh.pch, (int)sh.nch, false});
                    float ms = 0.f;
                    rc = time_step(ms, 6);
                    if (rc != NFM_OK) break;
                    timed.push_back({ms, sh});
                }
            }
        }
    }
    // the three fastest shapes again, twice with longer runs; the lowest time decides
    std::sort(timed.begin(), timed.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t i = 0; i < timed.size() && i < 3 && rc == NFM_OK; ++i) {
        const ChebShape& sh = timed[i].second;
        drop_entry();
        ctx->fwd_tuned.push_back({n_pairs, sh.threads, sh.group, sh.pch, (int)sh.nch, false});
        for (int trial = 0; trial < 2 && rc == NFM_OK; ++trial) {
            float ms = 0.f;
            rc = time_step(ms, 12);
            if (rc == NFM_OK && ms / 12 < best) {
                best = ms / 12;
                best_sh = sh;
            }
        }
    }
    drop_entry();
    if (rc == NFM_OK)
        ctx->fwd_tuned.push_back({n_pairs, best_sh.threads, best_sh.group, best_sh.pch, (int)best_sh.nch, false});
    // With NFM_ALGO_AUTO, the same step with the direct recurrence; the faster algorithm is kept.
    bool direct = false;
    if (rc == NFM_OK && algorithm == NFM_ALGO_AUTO && !ctx->points) {
        float t_direct = 0.f;
        ctx->algorithm = NFM_ALGO_DIRECT;
        rc = time_step(t_direct, 12);
        if (rc == NFM_OK) {
            direct = t_direct / 12 < best;
            ctx->fwd_tuned.back().direct = direct;
        }
    }
    ctx->algorithm = algorithm;
    ctx->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != NFM_OK) drop_entry();
    NFM_TRY(rc);
    NFM_TRY(check_flags(ctx));
    if (algorithm_out) *algorithm_out = direct ? NFM_ALGO_DIRECT : NFM_ALGO_CHEBYSHEV;
    if (group_out) *group_out = best_sh.group;
    if (threads_out) *threads_out = best_sh.threads;
    if (pairs_per_cta_out) *pairs_per_cta_out = best_sh.pch;
    if (chunks_out) *chunks_out = (int)best_sh.nch;
    return NFM_OK;
}

int nfm_set_forward_shape(nfm_ctx* ctx, int n_pairs, int algorithm, int threads, int lanes_per_group,
                          int pairs_per_cta, int chunks)
{
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1 || n_pairs > ctx->P) return fail(ctx, NFM_ERR_ARG, "n_pairs = %d outside [1, P]", n_pairs);
    if (ctx->cheb_L == 0 || !ctx->uniform) return fail(ctx, NFM_ERR_STATE, "the expansion is not available here");
    if (algorithm != NFM_ALGO_CHEBYSHEV && algorithm != NFM_ALGO_DIRECT)
        return fail(ctx, NFM_ERR_ARG, "algorithm must be NFM_ALGO_CHEBYSHEV or NFM_ALGO_DIRECT");
    if (threads != 64 && threads != 128) return fail(ctx, NFM_ERR_ARG, "threads must be 64 or 128");
    if (lanes_per_group != 4 && lanes_per_group != 8) return fail(ctx, NFM_ERR_ARG, "lanes_per_group must be 4 or 8");
    const int ng = threads / lanes_per_group;
    if (pairs_per_cta < 4 || pairs_per_cta > ng || (pairs_per_cta & (pairs_per_cta - 1)))
        return fail(ctx, NFM_ERR_ARG, "pairs_per_cta must be a power of two in [4, %d]", ng);
    if (chunks < 1 || chunks > ctx->gd.n_tiles) return fail(ctx, NFM_ERR_ARG, "chunks outside [1, %d]", ctx->gd.n_tiles);
    ChebShape sh;
    NFM_TRY(cheb_shape(ctx, n_pairs, threads, lanes_per_group, pairs_per_cta, 0.0, chunks, &sh));
    for (size_t i = 0; i < ctx->fwd_tuned.size(); ++i)
        if (ctx->fwd_tuned[i].n_pairs == n_pairs) {
            ctx->fwd_tuned.erase(ctx->fwd_tuned.begin() + i);
            break;
        }
    ctx->fwd_tuned.push_back({n_pairs, sh.threads, sh.group, sh.pch, (int)sh.nch, algorithm == NFM_ALGO_DIRECT});
    return NFM_OK;
}

int nfm_cheb_coefficients(double z_step, double k_center, int K, int L, double* out)
{
    if (K < 1 || L < 1 || L > 256 || !out || !std::isfinite(z_step) || !std::isfinite(k_center)) return NFM_ERR_ARG;
    cheb_coefficients(z_step, k_center, K, L, out);
    return NFM_OK;
}

int nfm_dims(const nfm_ctx* ctx, int* T, int* R, int* K, long long* N)
{
    if (!ctx || !ctx->has_geom) return NFM_ERR_STATE;
    if (T) *T = ctx->T;
    if (R) *R = ctx->R;
    if (K) *K = ctx->K;
    if (N) *N = ctx->N;
    return NFM_OK;
}

int nfm_forward(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* s, float* y)
{
    TraceRange trace_("nfm_forward");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1) return fail(ctx, NFM_ERR_ARG, "n_pairs must be >= 1");
    NFM_TRY(check_ptr(ctx, pairs, "pairs", 4));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    return enqueue_forward(ctx, pairs, n_pairs, (const float2*)s, nullptr, (float2*)y);
}

int nfm_residual(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* s, const float* y, float* r)
{
    TraceRange trace_("nfm_residual");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1) return fail(ctx, NFM_ERR_ARG, "n_pairs must be >= 1");
    NFM_TRY(check_ptr(ctx, pairs, "pairs", 4));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    NFM_TRY(check_ptr(ctx, r, "r", 8));
    return enqueue_forward(ctx, pairs, n_pairs, (const float2*)s, (const float2*)y, (float2*)r);
}

int nfm_adjoint(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* r, float* g)
{
    TraceRange trace_("nfm_adjoint");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1) return fail(ctx, NFM_ERR_ARG, "n_pairs must be >= 1");
    NFM_TRY(check_ptr(ctx, pairs, "pairs", 4));
    NFM_TRY(check_ptr(ctx, r, "r", 8));
    NFM_TRY(check_ptr(ctx, g, "g", 8));
    return enqueue_adjoint(ctx, pairs, n_pairs, (const float2*)r, (float2*)g, nullptr, 0.f, 0.f);
}

int nfm_spgm_step(nfm_ctx* ctx, const float* y, float* s, const int* pairs, int n_pairs, float eta, float lambda)
{
    TraceRange trace_("nfm_spgm_step");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1) return fail(ctx, NFM_ERR_ARG, "n_pairs must be >= 1");
    if (!(eta > 0) || !std::isfinite(eta)) return fail(ctx, NFM_ERR_ARG, "eta must be finite and > 0");
    if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(ctx, NFM_ERR_ARG, "lambda must be finite and >= 0");
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, pairs, "pairs", 4));
    return spgm_step_impl(ctx, (const float2*)y, (float2*)s, pairs, n_pairs, eta, lambda);
}

int nfm_spgm_epoch(nfm_ctx* ctx, const float* y, float* s, const int* perm, int pairs_per_batch, float eta,
                   float lambda)
{
    TraceRange trace_("nfm_spgm_epoch");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (pairs_per_batch < 1) return fail(ctx, NFM_ERR_ARG, "pairs_per_batch must be >= 1");
    if (!(eta > 0) || !std::isfinite(eta)) return fail(ctx, NFM_ERR_ARG, "eta must be finite and > 0");
    if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(ctx, NFM_ERR_ARG, "lambda must be finite and >= 0");
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, perm, "perm", 4));
    return spgm_epoch_impl(ctx, (const float2*)y, (float2*)s, perm, pairs_per_batch, eta, lambda);
}

int nfm_spgm_epochs_host(nfm_ctx* ctx, const float* y_host, float* s_host, const int* perms_host, int n_epochs,
                         int pairs_per_batch, float eta, float lambda)
{
    TraceRange trace_("nfm_spgm_epochs_host");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_epochs < 1 || pairs_per_batch < 1) return fail(ctx, NFM_ERR_ARG, "n_epochs and pairs_per_batch must be >= 1");
    if (!(eta > 0) || !std::isfinite(eta)) return fail(ctx, NFM_ERR_ARG, "eta must be finite and > 0");
    if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(ctx, NFM_ERR_ARG, "lambda must be finite and >= 0");
    if (!y_host || !s_host || !perms_host) return fail(ctx, NFM_ERR_ARG, "NULL host buffer");
    const size_t yb = (size_t)ctx->M * sizeof(float2), sb = (size_t)ctx->N * sizeof(float2);
    const size_t pb = (size_t)n_epochs * ctx->P * sizeof(int);
    NFM_TRY(ensure(ctx, &ctx->d_hy, &ctx->hy_cap, yb));
    NFM_TRY(ensure(ctx, &ctx->d_hs, &ctx->hs_cap, sb));
    NFM_TRY(ensure(ctx, &ctx->d_hperm, &ctx->hperm_cap, pb));
    NFM_CK(cudaMemcpyAsync(ctx->d_hy, y_host, yb, cudaMemcpyHostToDevice, ctx->stream));
    NFM_CK(cudaMemcpyAsync(ctx->d_hs, s_host, sb, cudaMemcpyHostToDevice, ctx->stream));
    NFM_CK(cudaMemcpyAsync(ctx->d_hperm, perms_host, pb, cudaMemcpyHostToDevice, ctx->stream));
    for (int e = 0; e < n_epochs; ++e)
        NFM_TRY(spgm_epoch_impl(ctx, (const float2*)ctx->d_hy, (float2*)ctx->d_hs,
                                (const int*)ctx->d_hperm + (size_t)e * ctx->P, pairs_per_batch, eta, lambda));
    NFM_CK(cudaMemcpyAsync(s_host, ctx->d_hs, sb, cudaMemcpyDeviceToHost, ctx->stream));
    NFM_CK(ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize());
    return check_flags(ctx);
}

int nfm_spgm_step_freqs(nfm_ctx* ctx, const float* y, float* s, const int* pairs, int n_pairs,
                        const unsigned char* freq_mask, int n_freq, float eta, float lambda)
{
    TraceRange trace_("nfm_spgm_step_freqs");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1) return fail(ctx, NFM_ERR_ARG, "n_pairs must be >= 1");
    if (n_freq < 1 || n_freq > ctx->K) return fail(ctx, NFM_ERR_ARG, "n_freq must be in [1, K]");
    if (!(eta > 0) || !std::isfinite(eta)) return fail(ctx, NFM_ERR_ARG, "eta must be finite and > 0");
    if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(ctx, NFM_ERR_ARG, "lambda must be finite and >= 0");
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, pairs, "pairs", 4));
    NFM_TRY(check_ptr(ctx, freq_mask, "freq_mask", 1));
    NFM_TRY(ensure(ctx, &ctx->d_resid, &ctx->resid_cap, (size_t)n_pairs * ctx->K * sizeof(float2)));
    float2* r = (float2*)ctx->d_resid;
    NFM_TRY(enqueue_forward(ctx, pairs, n_pairs, (const float2*)s, (const float2*)y, r, freq_mask));
    const double B = (double)n_pairs * n_freq;
    return enqueue_adjoint(ctx, pairs, n_pairs, r, nullptr, (float2*)s, (float)(eta / B),
                           (float)((double)eta * lambda * ctx->reg_w1),
                           (float)(1.0 / (1.0 + (double)eta * lambda * ctx->reg_w2)),
                           (float)((double)eta * lambda * ctx->reg_w3));
}

int nfm_pgm_step(nfm_ctx* ctx, const float* y, float* s, float eta, float lambda)
{
    TraceRange trace_("nfm_pgm_step");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (!(eta > 0) || !std::isfinite(eta)) return fail(ctx, NFM_ERR_ARG, "eta must be finite and > 0");
    if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(ctx, NFM_ERR_ARG, "lambda must be finite and >= 0");
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    return spgm_step_impl(ctx, (const float2*)y, (float2*)s, ctx->d_pairs_all, ctx->P, eta, lambda);
}

int nfm_solve(nfm_ctx* ctx, const float* y, float* s, const int* perms, int max_epochs, int pairs_per_batch,
              float eta, float lambda, double tol, int* epochs_out, double* change_out)
{
    TraceRange trace_("nfm_solve");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (max_epochs < 1 || pairs_per_batch < 1) return fail(ctx, NFM_ERR_ARG, "max_epochs and pairs_per_batch must be >= 1");
    if (!(eta > 0) || !std::isfinite(eta)) return fail(ctx, NFM_ERR_ARG, "eta must be finite and > 0");
    if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(ctx, NFM_ERR_ARG, "lambda must be finite and >= 0");
    if (!(tol >= 0)) return fail(ctx, NFM_ERR_ARG, "tol must be >= 0");
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, perms, "perms", 4));
    if (!epochs_out || !change_out) return fail(ctx, NFM_ERR_ARG, "NULL output");
    const size_t nb = (size_t)ctx->N * sizeof(float2);
    NFM_TRY(ensure(ctx, &ctx->d_v, &ctx->v_cap, nb));
    float2* prev = (float2*)ctx->d_v;
    double* part = ctx->d_red;
    double* sc = ctx->d_red + RED_BLOCKS;
    cudaStream_t st = ctx->stream;
    double change = 0.0;
    int e = 0;
    while (e < max_epochs) {
        NFM_CK(cudaMemcpyAsync(prev, s, nb, cudaMemcpyDeviceToDevice, st));
        NFM_TRY(spgm_epoch_impl(ctx, (const float2*)y, (float2*)s, perms + (size_t)e * ctx->P, pairs_per_batch,
                                eta, lambda));
        NFM_CK(launch_mag_change((const float2*)s, prev, ctx->N, part, sc + 0, st));
        NFM_CK(cudaMemcpyAsync(&change, sc + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
        NFM_CK(st ? cudaStreamSynchronize(st) : cudaDeviceSynchronize());
        ++e;
        if (change < tol) break;
    }
    NFM_TRY(check_flags(ctx));
    *epochs_out = e;
    *change_out = change;
    return NFM_OK;
}

int nfm_prox_step(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float shrink, long long n,
                  float* out)
{
    if (!ctx) return NFM_ERR_ARG;
    DevGuard guard(ctx->device);
    if (n < 1) return fail(ctx, NFM_ERR_ARG, "n must be >= 1");
    if (!std::isfinite(step) || !(alpha >= 0) || !std::isfinite(alpha) || !(shrink > 0) || !std::isfinite(shrink))
        return fail(ctx, NFM_ERR_ARG, "bad step/alpha/shrink");
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, g, "g", 8));
    NFM_TRY(check_ptr(ctx, out, "out", 8));
    NFM_CK(launch_prox_step((const float2*)s, (const float2*)g, step, alpha, shrink, n, (float2*)out, ctx->stream));
    return NFM_OK;
}

int nfm_prox_step_backward(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float shrink,
                           long long n, const float* grad_out, float* grad_s, float* grad_g, double* grad_scalars)
{
    if (!ctx) return NFM_ERR_ARG;
    DevGuard guard(ctx->device);
    if (n < 1) return fail(ctx, NFM_ERR_ARG, "n must be >= 1");
    if (!std::isfinite(step) || !(alpha >= 0) || !std::isfinite(alpha) || !(shrink > 0) || !std::isfinite(shrink))
        return fail(ctx, NFM_ERR_ARG, "bad step/alpha/shrink");
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, g, "g", 8));
    NFM_TRY(check_ptr(ctx, grad_out, "grad_out", 8));
    NFM_TRY(check_ptr(ctx, grad_scalars, "grad_scalars", 8));
    if (grad_s) NFM_TRY(check_ptr(ctx, grad_s, "grad_s", 8));
    if (grad_g) NFM_TRY(check_ptr(ctx, grad_g, "grad_g", 8));
    NFM_TRY(ensure(ctx, &ctx->d_prox_partial, &ctx->prox_partial_cap, 3 * RED_BLOCKS * sizeof(double)));
    NFM_CK(launch_prox_step_backward((const float2*)s, (const float2*)g, step, alpha, shrink, n, (const float2*)grad_out,
                                     (float2*)grad_s, (float2*)grad_g, (double*)ctx->d_prox_partial, grad_scalars,
                                     ctx->stream));
    return NFM_OK;
}

int nfm_prox_group_step(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float alpha_g,
                        float shrink, float* out)
{
    if (!ctx) return NFM_ERR_ARG;
    TraceRange trace_("nfm_prox_group_step");
    DevGuard guard(ctx->device);
    NFM_TRY(require_geom(ctx));
    if (ctx->points) return fail(ctx, NFM_ERR_STATE, "the group term of the regulariser needs a regular voxel grid");
    if (!std::isfinite(step) || !(alpha >= 0) || !std::isfinite(alpha) || !(alpha_g >= 0) || !std::isfinite(alpha_g) ||
        !(shrink > 0) || !std::isfinite(shrink))
        return fail(ctx, NFM_ERR_ARG, "bad step/alpha/alpha_g/shrink");
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, g, "g", 8));
    NFM_TRY(check_ptr(ctx, out, "out", 8));
    NFM_CK(launch_prox_group_step((const float2*)s, (const float2*)g, step, alpha, alpha_g, shrink, ctx->gd.nx,
                                  ctx->gd.ny, ctx->gd.nz, (float2*)out, ctx->stream));
    return NFM_OK;
}

int nfm_prox_group_step_backward(nfm_ctx* ctx, const float* s, const float* g, float step, float alpha, float alpha_g,
                                 float shrink, const float* grad_out, float* grad_s, float* grad_g,
                                 double* grad_scalars)
{
    if (!ctx) return NFM_ERR_ARG;
    TraceRange trace_("nfm_prox_group_step_backward");
    DevGuard guard(ctx->device);
    NFM_TRY(require_geom(ctx));
    if (ctx->points) return fail(ctx, NFM_ERR_STATE, "the group term of the regulariser needs a regular voxel grid");
    if (!std::isfinite(step) || !(alpha >= 0) || !std::isfinite(alpha) || !(alpha_g >= 0) || !std::isfinite(alpha_g) ||
        !(shrink > 0) || !std::isfinite(shrink))
        return fail(ctx, NFM_ERR_ARG, "bad step/alpha/alpha_g/shrink");
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, g, "g", 8));
    NFM_TRY(check_ptr(ctx, grad_out, "grad_out", 8));
    NFM_TRY(check_ptr(ctx, grad_scalars, "grad_scalars", 8));
    if (grad_s) NFM_TRY(check_ptr(ctx, grad_s, "grad_s", 8));
    if (grad_g) NFM_TRY(check_ptr(ctx, grad_g, "grad_g", 8));
    NFM_TRY(ensure(ctx, &ctx->d_prox_partial, &ctx->prox_partial_cap, 4 * RED_BLOCKS * sizeof(double)));
    NFM_CK(launch_prox_group_step_backward((const float2*)s, (const float2*)g, step, alpha, alpha_g, shrink,
                                           ctx->gd.nx, ctx->gd.ny, ctx->gd.nz, (const float2*)grad_out,
                                           (float2*)grad_s, (float2*)grad_g, (double*)ctx->d_prox_partial,
                                           grad_scalars, ctx->stream));
    return NFM_OK;
}

}  // extern "C"

namespace {
// lambda_max(A_B^H A_B) / B for the rows of the listed pairs (B = n_pairs K) by `iters` power
// iterations from v0, FP64 norms (the full operator is the list of every pair)
int power_iteration_impl(nfm_ctx* ctx, const int* pairs, int n_pairs, int iters, const float* v0, double* L_out)
{
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (iters < 0) return fail(ctx, NFM_ERR_ARG, "iters must be >= 0");
    NFM_TRY(check_ptr(ctx, v0, "v0", 8));
    if (!L_out) return fail(ctx, NFM_ERR_ARG, "L_out is NULL");
    const long long rows = (long long)n_pairs * ctx->K;
    const size_t nb = (size_t)ctx->N * sizeof(float2), mb = (size_t)rows * sizeof(float2);
    NFM_TRY(ensure(ctx, &ctx->d_v, &ctx->v_cap, nb));
    NFM_TRY(ensure(ctx, &ctx->d_g, &ctx->g_cap, nb));
    NFM_TRY(ensure(ctx, &ctx->d_y, &ctx->y_cap, mb));
    float2* v = (float2*)ctx->d_v;
    float2* g = (float2*)ctx->d_g;
    float2* y = (float2*)ctx->d_y;
    double* part = ctx->d_red;
    double* sc = ctx->d_red + RED_BLOCKS;   // scalars
    cudaStream_t st = ctx->stream;
    NFM_CK(launch_norm2((const float2*)v0, ctx->N, part, sc + 0, st));
    NFM_CK(launch_normalize((const float2*)v0, v, ctx->N, sc + 0, st));
    for (int it = 0; it < iters; ++it) {
        NFM_TRY(enqueue_forward(ctx, pairs, n_pairs, v, nullptr, y));
        NFM_TRY(enqueue_adjoint(ctx, pairs, n_pairs, y, g, nullptr, 0.f, 0.f));
        const int e0 = prof_mark(ctx);
        NFM_CK(launch_norm2(g, ctx->N, part, sc + 0, st));
        NFM_CK(launch_normalize(g, v, ctx->N, sc + 0, st));
        prof_pair(ctx, 3, e0, prof_mark(ctx));
    }
    NFM_TRY(enqueue_forward(ctx, pairs, n_pairs, v, nullptr, y));
    NFM_CK(launch_norm2(y, rows, part, sc + 1, st));
    NFM_CK(launch_norm2(v, ctx->N, part, sc + 2, st));
    NFM_CK(launch_ratio(sc + 1, sc + 2, (double)rows, sc + 3, st));
    double L = 0;
    NFM_CK(cudaMemcpyAsync(&L, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    NFM_CK(st ? cudaStreamSynchronize(st) : cudaDeviceSynchronize());
    NFM_TRY(check_flags(ctx));
    if (!std::isfinite(L)) return fail(ctx, NFM_ERR_NUMERIC, "power iteration gave a non-finite L");
    *L_out = L;
    return NFM_OK;
}
}  // namespace

extern "C" {

int nfm_power_iteration(nfm_ctx* ctx, int iters, const float* v0, double* L_out)
{
    TraceRange trace_("nfm_power_iteration");
    NFM_TRY(require_geom(ctx));
    return power_iteration_impl(ctx, ctx->d_pairs_all, ctx->P, iters, v0, L_out);
}

int nfm_power_iteration_pairs(nfm_ctx* ctx, const int* pairs, int n_pairs, int iters, const float* v0,
                              double* L_out)
{
    TraceRange trace_("nfm_power_iteration_pairs");
    NFM_TRY(require_geom(ctx));
    if (n_pairs < 1) return fail(ctx, NFM_ERR_ARG, "n_pairs must be >= 1");
    NFM_TRY(check_ptr(ctx, pairs, "pairs", 4));
    return power_iteration_impl(ctx, pairs, n_pairs, iters, v0, L_out);
}

int nfm_objective(nfm_ctx* ctx, const float* y, const float* s, double lambda, double* F_out)
{
    TraceRange trace_("nfm_objective");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    if (!F_out) return fail(ctx, NFM_ERR_ARG, "F_out is NULL");
    const size_t mb = (size_t)ctx->M * sizeof(float2);
    NFM_TRY(ensure(ctx, &ctx->d_y, &ctx->y_cap, mb));
    float2* res = (float2*)ctx->d_y;
    double* part = ctx->d_red;
    double* sc = ctx->d_red + RED_BLOCKS;
    cudaStream_t st = ctx->stream;
    NFM_TRY(enqueue_forward(ctx, ctx->d_pairs_all, ctx->P, (const float2*)s, (const float2*)y, res));
    NFM_CK(launch_norm2(res, ctx->M, part, sc + 4, st));
    NFM_CK(launch_abs_sum((const float2*)s, ctx->N, part, sc + 5, st));
    NFM_CK(launch_axpby(sc + 4, 1.0 / (2.0 * (double)ctx->M), sc + 5, lambda * ctx->reg_w1, sc + 6, st));
    double F = 0, s2 = 0, gsum = 0;
    NFM_CK(cudaMemcpyAsync(&F, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (ctx->reg_w2 != 0.0) {
        NFM_CK(launch_norm2((const float2*)s, ctx->N, part, sc + 2, st));
        NFM_CK(cudaMemcpyAsync(&s2, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (ctx->reg_w3 != 0.0) {
        if (ctx->points) return fail(ctx, NFM_ERR_ARG, "the group term of the regulariser needs a regular voxel grid");
        NFM_CK(launch_group_norm_sum((const float2*)s, ctx->gd.nx, ctx->gd.ny, ctx->gd.nz, part, sc + 3, st));
        NFM_CK(cudaMemcpyAsync(&gsum, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    NFM_CK(st ? cudaStreamSynchronize(st) : cudaDeviceSynchronize());
    NFM_TRY(check_flags(ctx));
    *F_out = F + 0.5 * lambda * ctx->reg_w2 * s2 + lambda * ctx->reg_w3 * gsum;
    return NFM_OK;
}

int nfm_lambda_max(nfm_ctx* ctx, const float* y, double* out)
{
    TraceRange trace_("nfm_lambda_max");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    if (!out) return fail(ctx, NFM_ERR_ARG, "out is NULL");
    const size_t nb = (size_t)ctx->N * sizeof(float2);
    NFM_TRY(ensure(ctx, &ctx->d_g, &ctx->g_cap, nb));
    double* part = ctx->d_red;
    double* sc = ctx->d_red + RED_BLOCKS;
    cudaStream_t st = ctx->stream;
    NFM_TRY(enqueue_adjoint(ctx, ctx->d_pairs_all, ctx->P, (const float2*)y, (float2*)ctx->d_g, nullptr, 0.f, 0.f));
    NFM_CK(launch_abs_max((const float2*)ctx->d_g, ctx->N, part, sc + 7, st));
    double m = 0;
    NFM_CK(cudaMemcpyAsync(&m, sc + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
    NFM_CK(st ? cudaStreamSynchronize(st) : cudaDeviceSynchronize());
    NFM_TRY(check_flags(ctx));
    *out = m / (double)ctx->M;
    return NFM_OK;
}

int nfm_synchronize(nfm_ctx* ctx)
{
    if (!ctx) return NFM_ERR_ARG;
    DevGuard guard(ctx->device);
    NFM_CK(ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize());
    return check_flags(ctx);
}

static_assert((int)NFM_HOOK_TC_SKIP_ISSUE == (int)HOOK_TC_SKIP_ISSUE, "hook flags of the header and the kernels");
static_assert((int)NFM_HOOK_SHRINK_EXTENTS == (int)HOOK_SHRINK_EXTENTS, "hook flags of the header and the kernels");

int nfm_set_test_hooks(nfm_ctx* ctx, int flags, int wait_ms)
{
    if (!ctx) return NFM_ERR_ARG;
    if (flags & ~(NFM_HOOK_TC_SKIP_ISSUE | NFM_HOOK_SHRINK_EXTENTS))
        return fail(ctx, NFM_ERR_ARG, "unknown test hook flags 0x%x", flags);
    if (wait_ms < 0 || wait_ms > 60000) return fail(ctx, NFM_ERR_ARG, "wait_ms must lie in [0, 60000]");
    ctx->hooks = flags;
    ctx->tc_wait_ns = wait_ms > 0 ? (unsigned long long)wait_ms * 1000000ull : 1000000000ull;
    return NFM_OK;
}

int nfm_profile_enable(nfm_ctx* ctx, int enable)
{
    if (!ctx) return NFM_ERR_ARG;
    ctx->prof = enable != 0;
    return NFM_OK;
}

int nfm_profile_report(nfm_ctx* ctx, double* ms_out, long long* launches_out, int n_kinds)
{
    if (!ctx) return NFM_ERR_ARG;
    if (n_kinds < 0 || (n_kinds > 0 && (!ms_out || !launches_out)))
        return fail(ctx, NFM_ERR_ARG, "bad output arrays");
    DevGuard guard(ctx->device);
    NFM_CK(ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize());
    for (int i = 0; i < n_kinds; ++i) {
        ms_out[i] = 0.0;
        launches_out[i] = 0;
    }
    for (const auto& p : ctx->pending) {
        float ms = 0.f;
        NFM_CK(cudaEventElapsedTime(&ms, ctx->ev_pool[p.a], ctx->ev_pool[p.b]));
        if (p.kind < n_kinds) {
            ms_out[p.kind] += ms;
            launches_out[p.kind] += 1;
        }
    }
    ctx->pending.clear();
    ctx->ev_used = 0;
    return NFM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free forward: the chunk partial sums live in a static device
// array instead of library-owned cudaMalloc scratch.  Nothing here allocates.
namespace {
constexpr size_t NOALLOC_SCRATCH_ELEMS = (size_t)1 << 19;   // complex64 partial sums, 4 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;
}  // namespace

static __device__ __align__(256) float2 g_noalloc_scratch[NOALLOC_SCRATCH_ELEMS];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on ctx->device (looked up once per
// device, with that device current; the caller holds a DevGuard).
int noalloc_scratch(nfm_ctx* ctx, float2** out)
{
    if (ctx->device < 0 || ctx->device >= NOALLOC_MAX_DEVICES)
        return fail(ctx, NFM_ERR_ARG, "device %d: the allocation-free path supports devices 0..%d", ctx->device,
                    NOALLOC_MAX_DEVICES - 1);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, NFM_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        g_noalloc_addr[ctx->device] = p;
    }
    *out = (float2*)g_noalloc_addr[ctx->device];
    return NFM_OK;
}
}  // namespace

extern "C" int nfm_forward_noalloc(nfm_ctx* ctx, const int* pairs, int n_pairs, const float* s, float* y)
{
    TraceRange trace_("nfm_forward_noalloc");
    NFM_TRY(require_geom(ctx));
    DevGuard guard(ctx->device);
    if (n_pairs < 1) return fail(ctx, NFM_ERR_ARG, "n_pairs must be >= 1");
    NFM_TRY(check_ptr(ctx, pairs, "pairs", 4));
    NFM_TRY(check_ptr(ctx, s, "s", 8));
    NFM_TRY(check_ptr(ctx, y, "y", 8));
    if (!ctx->uniform)
        return fail(ctx, NFM_ERR_ARG, "the allocation-free forward needs equally spaced frequencies");
    if (ctx->points) return fail(ctx, NFM_ERR_ARG, "the allocation-free forward needs a regular voxel grid");
    // one voxel chunk holds ceil(n_pairs / 8) * 8 * K partial sums (pairs padded to whole CTAs)
    const size_t per_chunk = (size_t)((n_pairs + FWD_PC - 1) / FWD_PC) * FWD_PC * ctx->K;
    if (per_chunk > NOALLOC_SCRATCH_ELEMS)
        return fail(ctx, NFM_ERR_ARG, "ceil(n_pairs / 8) * 8 * K = %zu exceeds the allocation-free limit %zu",
                    per_chunk, NOALLOC_SCRATCH_ELEMS);
    FwdPlan pl;
    NFM_TRY(plan_forward(ctx, n_pairs, &pl, (long long)(NOALLOC_SCRATCH_ELEMS / per_chunk)));
    float2* scratch = nullptr;
    NFM_TRY(noalloc_scratch(ctx, &scratch));
    OpDesc op = op_desc(ctx);
    FwdArgs a;
    a.pairs = pairs;
    a.n_pairs = n_pairs;
    a.s = (const float2*)s;
    a.partial = scratch;
    a.partial_elems = (long long)NOALLOC_SCRATCH_ELEMS;
    a.n_slots = pl.n_slots;
    a.VS = pl.VS;
    a.tiles_base = pl.base;
    a.tiles_rem = pl.rem;
    NFM_CK(launch_fwd_partial(op, a, dim3(pl.n_groups, pl.n_chunks), pl.nt, pl.smem, ctx->stream));
    ReduceArgs ra;
    ra.partial = scratch;
    ra.partial_elems = (long long)NOALLOC_SCRATCH_ELEMS / ((ctx->hooks & HOOK_SHRINK_EXTENTS) ? 2 : 1);
    ra.n_chunks = pl.n_chunks;
    ra.n_slots = pl.n_slots;
    ra.n_out = n_pairs * ctx->K;
    ra.pairs = pairs;
    ra.y_obs = nullptr;
    ra.fmask = nullptr;
    ra.out = (float2*)y;
    NFM_CK(launch_fwd_reduce(op, ra, ctx->stream));
    return NFM_OK;
}

// ---------------------------------------------------------------------------
// Batched scenes: one CUDA graph per epoch with a concurrent branch per scene.
struct nfm_batch {
    std::vector<nfm_ctx*> scenes;
    cudaStream_t stream = nullptr;          // caller's stream (graph launches)
    cudaStream_t cap = nullptr;             // capture origin
    std::vector<cudaStream_t> branch;       // one per scene
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    // arguments of the captured call
    std::vector<const void*> y, s, perm;
    std::vector<int> bp;
    std::vector<float> eta, lam;
    std::vector<unsigned long long> gen;   // scene scratch generations the graph was captured with
    std::string err;
    int mode = NFM_BATCH_BRANCHES;
    int captured_mode = -1;
    // fused mode: scene items of every launch and the coefficient tables padded to the launch's L
    void* d_items = nullptr;
    std::vector<float*> d_coef;
};

namespace {

int bfail(nfm_batch* b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    b->err = buf;
    return code;
}

#define NFM_BCK(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail(b, NFM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

// Allocate and plan everything an epoch of this scene needs, so that the capture
// performs no allocation.
int prepare_epoch(nfm_ctx* ctx, int bp)
{
    NFM_TRY(ensure(ctx, &ctx->d_resid, &ctx->resid_cap, (size_t)bp * ctx->K * sizeof(float2)));
    for (int nb : {bp, ctx->P % bp}) {
        if (nb <= 0) continue;
        FwdPlan pl;
        size_t pbytes = 0;
        bool cheb = false;
        if (ctx->uniform) NFM_TRY(use_cheb(ctx, cheb, nb));
        if (!ctx->uniform) {
            plan_forward_general(ctx, nb, &pl);
            pbytes = pl.partial_bytes;
        } else if (cheb && ctx->precision != NFM_FP32) {       // the tensor-core forward's shape
            int pch = 0, ng = 0;
            long long nch = 0;
            tc_fwd_shape(ctx, nb, &pch, &ng, &nch);
            pbytes = (size_t)nch * ng * pch * ctx->K * sizeof(float2);
        } else if (cheb) {                                      // the expansion forward's (tuned or default) shape
            ChebShape sh;
            bool tuned = false;
            for (const auto& t : ctx->fwd_tuned)
                if (t.n_pairs == nb && !t.direct) {
                    NFM_TRY(cheb_shape(ctx, nb, t.threads, t.group, t.pch, 0.0, t.chunks, &sh));
                    tuned = true;
                }
            if (!tuned) NFM_TRY(cheb_shape(ctx, nb, CHEB_THREADS, CHEB_GROUP, 0, 2.0, 0, &sh));
            pbytes = (size_t)sh.nch * sh.n_slots * ctx->K * sizeof(float2);
        } else {
            NFM_TRY(plan_forward(ctx, nb, &pl));
            pbytes = pl.partial_bytes;
        }
        NFM_TRY(ensure(ctx, &ctx->d_partial, &ctx->partial_cap, pbytes));
        if (ctx->precision != NFM_FP32) {
            NFM_TRY(ensure(ctx, &ctx->d_bmat, &ctx->bmat_cap, adj_tc_bmat_bytes(nb)));
            NFM_TRY(ensure(ctx, &ctx->d_bscale, &ctx->bscale_cap, (size_t)nb * sizeof(float)));
        }
    }
    const int K1 = ctx->K1;
    if (ctx->precision == NFM_FP32 && !ctx->adj_attr[K1]) {
        NFM_CK(cudaFuncSetAttribute(adj_kernel_ptr(K1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ctx->smem_optin));
        ctx->adj_attr[K1] = true;
    }
    if (ctx->precision != NFM_FP32) {
        const bool f16 = ctx->precision == NFM_TC_FP16X3;
        if (!ctx->adj_tc_attr[f16][K1]) {
            NFM_CK(cudaFuncSetAttribute(adj_tc_kernel_ptr(K1, f16), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ctx->smem_optin));
            ctx->adj_tc_attr[f16][K1] = true;
        }
    }
    return NFM_OK;
}

}  // namespace

extern "C" {

int nfm_batch_create(nfm_batch** out, nfm_ctx* const* scenes, int n_scenes, void* cuda_stream)
{
    if (!out) return NFM_ERR_ARG;
    *out = nullptr;
    if (!scenes || n_scenes < 1) return fail(nullptr, NFM_ERR_ARG, "need at least one scene");
    for (int i = 0; i < n_scenes; ++i)
        if (!scenes[i]) return fail(nullptr, NFM_ERR_ARG, "scene %d is NULL", i);
    const int dev = scenes[0]->device;
    for (int i = 1; i < n_scenes; ++i)
        if (scenes[i]->device != dev) return fail(nullptr, NFM_ERR_ARG, "all scenes must be on one device");
    DevGuard guard(dev);
    nfm_batch* b = new nfm_batch();
    b->scenes.assign(scenes, scenes + n_scenes);
    b->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    b->branch.assign(n_scenes, nullptr);
    b->join.assign(n_scenes, nullptr);
    for (int i = 0; i < n_scenes && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        nfm_batch_destroy(b);
        return fail(nullptr, NFM_ERR_CUDA, "batch streams/events: %s", cudaGetErrorString(e));
    }
    *out = b;
    return NFM_OK;
}

void nfm_batch_destroy(nfm_batch* b)
{
    if (!b) return;
    DevGuard guard(b->scenes.empty() ? 0 : b->scenes[0]->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t st : b->branch)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    free_ptr(b->d_items);
    for (float* p : b->d_coef) free_ptr(p);
    delete b;
}

const char* nfm_batch_last_error(const nfm_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int nfm_batch_set_mode(nfm_batch* b, int mode)
{
    if (!b) return NFM_ERR_ARG;
    if (mode != NFM_BATCH_BRANCHES && mode != NFM_BATCH_FUSED) return bfail(b, NFM_ERR_ARG, "unknown batch mode %d", mode);
    b->mode = mode;
    return NFM_OK;
}

}  // extern "C"

namespace {

// Fused epoch: for step t of the epoch, one launch each of the expansion forward, the chunk reduction and
// the expansion adjoint over every scene that still has a minibatch at t (scene i takes pairs
// perm_i[t bp_i ...]), enqueued on `st` (the capture stream).
int batch_fused_enqueue(nfm_batch* b, const float* const* y, float* const* s, const int* const* perm,
                        const int* bp, const float* eta, const float* lambda, cudaStream_t st)
{
    const int n = (int)b->scenes.size();
    int LT = 0, steps = 0;
    for (int i = 0; i < n; ++i) {
        nfm_ctx* c = b->scenes[i];
        if (!c->uniform || c->cheb_L == 0 || c->algorithm == NFM_ALGO_DIRECT || c->precision != NFM_FP32)
            return bfail(b, NFM_ERR_ARG, "scene %d: the fused batch needs the FP32 expansion operator", i);
        LT = std::max(LT, c->cheb_L);
        steps = std::max(steps, (c->P + bp[i] - 1) / bp[i]);
    }
    if (!fwd_cheb_multi_ptr(LT))
        return bfail(b, NFM_ERR_ARG, "the fused batch covers expansion lengths up to 20 (here %d)", LT);
    const int LS = (LT + 3) & ~3;
    // coefficient tables with the row stride of LT (zero columns beyond each scene's L)
    for (float* p : b->d_coef) free_ptr(p);
    b->d_coef.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        nfm_ctx* c = b->scenes[i];
        const size_t bytes = (size_t)c->cheb_kpad * LS * sizeof(float);
        cudaError_t e = cudaMalloc((void**)&b->d_coef[i], bytes);
        if (e == cudaSuccess) e = cudaMemset(b->d_coef[i], 0, bytes);
        const int ls_i = (c->cheb_L + 3) & ~3;
        if (e == cudaSuccess)
            e = cudaMemcpy2D(b->d_coef[i], LS * sizeof(float), c->d_cheb, ls_i * sizeof(float), ls_i * sizeof(float),
                             c->cheb_kpad, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) return bfail(b, NFM_ERR_CUDA, "fused coefficient tables: %s", cudaGetErrorString(e));
    }
    std::vector<MultiFwdItem> fwd;
    std::vector<MultiRedItem> red;
    std::vector<MultiAdjItem> adj;
    struct Launch { size_t f0, nf, r0, nr, a0, na; int cf, cr, ca; };
    std::vector<Launch> launches;
    size_t smem_f = 0, smem_a = 0;
    for (int t = 0; t < steps; ++t) {
        Launch L{fwd.size(), 0, red.size(), 0, adj.size(), 0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            nfm_ctx* c = b->scenes[i];
            if (t * bp[i] >= c->P) continue;
            const int np = std::min(bp[i], c->P - t * bp[i]);
            const int* pairs = perm[i] + (size_t)t * bp[i];
            ChebShape sh;
            bool tuned = false;
            for (const auto& tu : c->fwd_tuned)
                if (tu.n_pairs == np && tu.threads == CHEB_THREADS && tu.group == CHEB_GROUP) {
                    NFM_TRY(cheb_shape(c, np, tu.threads, tu.group, tu.pch, 0.0, tu.chunks, &sh, true));
                    tuned = true;
                }
            if (!tuned) NFM_TRY(cheb_shape(c, np, CHEB_THREADS, CHEB_GROUP, 0, 2.0, 0, &sh, true));
            const size_t pbytes = (size_t)sh.nch * sh.n_slots * c->K * sizeof(float2);
            NFM_TRY(ensure(c, &c->d_partial, &c->partial_cap, pbytes));
            NFM_TRY(ensure(c, &c->d_resid, &c->resid_cap, (size_t)bp[i] * c->K * sizeof(float2)));
            smem_f = std::max(smem_f, fwd_cheb_smem_bytes(LT, c->cheb_kpad, sh.pch, CHEB_THREADS, CHEB_GROUP, c->points));
            smem_a = std::max(smem_a, adj_cheb_smem_bytes(LT, c->cheb_kpad));
            const OpDesc op = op_desc(c);
            ChebDesc cd{b->d_coef[i], c->cheb_tau, LT, c->cheb_kpad, c->cheb_fc_hi, c->cheb_fc_lo};
            MultiFwdItem fi;
            fi.op = op;
            fi.cd = cd;
            fi.a.pairs = pairs;
            fi.a.n_pairs = np;
            fi.a.s = (const float2*)s[i];
            fi.a.partial = (float2*)c->d_partial;
            fi.a.partial_elems = (long long)(c->partial_cap / sizeof(float2));
            fi.a.n_slots = sh.n_slots;
            fi.a.VS = sh.pch;
            fi.a.tiles_base = (int)(c->gd.n_tiles / sh.nch);
            fi.a.tiles_rem = (int)(c->gd.n_tiles % sh.nch);
            fi.n_groups = sh.n_groups;
            fi.cta0 = L.cf;
            L.cf += (int)(sh.n_groups * sh.nch);
            fwd.push_back(fi);
            MultiRedItem ri;
            ri.op = op;
            ri.a.partial = (const float2*)c->d_partial;
            ri.a.partial_elems = fi.a.partial_elems;
            ri.a.n_chunks = (int)sh.nch;
            ri.a.n_slots = sh.n_slots;
            ri.a.n_out = np * c->K;
            ri.a.pairs = pairs;
            ri.a.y_obs = (const float2*)y[i];
            ri.a.fmask = nullptr;
            ri.a.out = (float2*)c->d_resid;
            ri.cta0 = L.cr;
            L.cr += fwd_reduce_blocks(ri.a.n_out);
            red.push_back(ri);
            const double B = (double)np * c->K;
            MultiAdjItem ai;
            ai.op = op;
            ai.cd = cd;
            ai.a.pairs = pairs;
            ai.a.n_pairs = np;
            ai.a.r = (const float2*)c->d_resid;
            ai.a.r_elems = (long long)np * c->K;
            ai.a.g_out = nullptr;
            ai.a.s = (float2*)s[i];
            ai.a.step = (float)(eta[i] / B);
            ai.a.alpha = (float)((double)eta[i] * lambda[i] * c->reg_w1);
            ai.a.shrink = (float)(1.0 / (1.0 + (double)eta[i] * lambda[i] * c->reg_w2));
            ai.a.alpha_g = (float)((double)eta[i] * lambda[i] * c->reg_w3);
            ai.a.pchunk = CHEB_ADJ_PCHUNK;
            ai.cta0 = L.ca;
            L.ca += c->gd.n_tiles;
            adj.push_back(ai);
        }
        L.nf = fwd.size() - L.f0;
        L.nr = red.size() - L.r0;
        L.na = adj.size() - L.a0;
        launches.push_back(L);
    }
    for (nfm_ctx* c : b->scenes)
        if (c->points && c->reg_w3 != 0.0) return bfail(b, NFM_ERR_ARG, "the group term needs a regular voxel grid");
    // every item of every launch in one device buffer
    const size_t bf = fwd.size() * sizeof(MultiFwdItem), br = red.size() * sizeof(MultiRedItem),
                 ba = adj.size() * sizeof(MultiAdjItem);
    free_ptr(b->d_items);
    b->d_items = nullptr;
    cudaError_t e = cudaMalloc(&b->d_items, bf + br + ba);
    unsigned char* base = (unsigned char*)b->d_items;
    if (e == cudaSuccess) e = cudaMemcpy(base, fwd.data(), bf, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + bf, red.data(), br, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + bf + br, adj.data(), ba, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fwd_cheb_multi_ptr(LT), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(adj_cheb_multi_ptr(LT), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
    if (e != cudaSuccess) return bfail(b, NFM_ERR_CUDA, "fused batch items: %s", cudaGetErrorString(e));
    const MultiFwdItem* df = (const MultiFwdItem*)base;
    const MultiRedItem* dr = (const MultiRedItem*)(base + bf);
    const MultiAdjItem* da = (const MultiAdjItem*)(base + bf + br);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    for (const Launch& L : launches) {
        if (e == cudaSuccess) e = launch_fwd_cheb_multi(LT, df + L.f0, (int)L.nf, L.cf, smem_f, st);
        if (e == cudaSuccess) e = launch_fwd_reduce_multi(dr + L.r0, (int)L.nr, L.cr, st);
        if (e == cudaSuccess) e = launch_adj_cheb_multi(LT, da + L.a0, (int)L.na, L.ca, smem_a, st);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(b, NFM_ERR_CUDA, "fused capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return bfail(b, NFM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    return NFM_OK;
}

}  // namespace

extern "C" {

int nfm_batch_spgm_epoch(nfm_batch* b, const float* const* y, float* const* s, const int* const* perm,
                         const int* pairs_per_batch, const float* eta, const float* lambda)
{
    TraceRange trace_("nfm_batch_spgm_epoch");
    if (!b) return NFM_ERR_ARG;
    const int n = (int)b->scenes.size();
    if (!y || !s || !perm || !pairs_per_batch || !eta || !lambda) return bfail(b, NFM_ERR_ARG, "NULL argument array");
    DevGuard guard(b->scenes[0]->device);
    bool same = b->exec != nullptr && b->captured_mode == b->mode;
    for (int i = 0; i < n; ++i) {
        nfm_ctx* c = b->scenes[i];
        if (!c->has_geom) return bfail(b, NFM_ERR_STATE, "scene %d has no geometry", i);
        if (c->prof) return bfail(b, NFM_ERR_STATE, "scene %d has profiling enabled", i);
        if (pairs_per_batch[i] < 1) return bfail(b, NFM_ERR_ARG, "scene %d: pairs_per_batch < 1", i);
        if (!(eta[i] > 0) || !std::isfinite(eta[i]) || !(lambda[i] >= 0) || !std::isfinite(lambda[i]))
            return bfail(b, NFM_ERR_ARG, "scene %d: bad eta/lambda", i);
        if (!y[i] || !s[i] || !perm[i]) return bfail(b, NFM_ERR_ARG, "scene %d: NULL vector", i);
        if (same && (b->y[i] != y[i] || b->s[i] != s[i] || b->perm[i] != perm[i] || b->bp[i] != pairs_per_batch[i] ||
                     b->eta[i] != eta[i] || b->lam[i] != lambda[i] || b->gen[i] != c->scratch_gen))
            same = false;
    }
    if (!same) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        for (int i = 0; i < n; ++i) {
            int r = prepare_epoch(b->scenes[i], pairs_per_batch[i]);
            if (r != NFM_OK) return bfail(b, r, "scene %d: %s", i, b->scenes[i]->err.c_str());
        }
        if (b->mode == NFM_BATCH_FUSED) {
            int r = batch_fused_enqueue(b, y, s, perm, pairs_per_batch, eta, lambda, b->cap);
            if (r != NFM_OK) return r;
        }
    }
    if (!same && b->mode == NFM_BATCH_BRANCHES) {
        NFM_BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        int rc = NFM_OK;
        cudaError_t e = cudaEventRecord(b->fork, b->cap);
        for (int i = 0; i < n && e == cudaSuccess && rc == NFM_OK; ++i) {
            nfm_ctx* c = b->scenes[i];
            e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
            if (e != cudaSuccess) break;
            cudaStream_t saved = c->stream;
            c->stream = b->branch[i];
            rc = spgm_epoch_impl(c, (const float2*)y[i], (float2*)s[i], perm[i], pairs_per_batch[i], eta[i], lambda[i]);
            c->stream = saved;
            if (rc != NFM_OK) break;
            e = cudaEventRecord(b->join[i], b->branch[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[i], 0);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
        if (rc != NFM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return bfail(b, rc, "capture: %s", b->scenes[0]->err.c_str());
        }
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bfail(b, NFM_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return bfail(b, NFM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
    }
    if (!same) {
        b->y.assign(y, y + n);
        b->s.assign((const void* const*)s, (const void* const*)s + n);
        b->perm.assign((const void* const*)perm, (const void* const*)perm + n);
        b->bp.assign(pairs_per_batch, pairs_per_batch + n);
        b->eta.assign(eta, eta + n);
        b->lam.assign(lambda, lambda + n);
        b->gen.resize(n);
        for (int i = 0; i < n; ++i) b->gen[i] = b->scenes[i]->scratch_gen;
        b->captured_mode = b->mode;
    }
    NFM_BCK(cudaGraphLaunch(b->exec, b->stream));
    return NFM_OK;
}

}  // extern "C"
