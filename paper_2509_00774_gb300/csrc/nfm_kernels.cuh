// Kernel argument blocks and host-side launch helpers shared by the
// translation units of the library.
#pragma once
#include "nfm_device.cuh"

namespace nfm {

struct FwdArgs {
    const int* pairs;        // [n_pairs] pair indices (device)
    int n_pairs;
    const float2* s;         // [N]
    float2* partial;         // [n_chunks][n_slots][K]
    int n_slots;             // n_groups * FWD_PC
    int VS;                  // voxel subsets per CTA
    int tiles_base;          // chunk c owns tiles_base (+1 for c < tiles_rem) tiles
    int tiles_rem;
    long long partial_elems = 0;   // extent of partial (checked in the bounds-checked build)
};

struct ReduceArgs {
    const float2* partial;   // [n_chunks][n_slots][K]
    int n_chunks;
    int n_slots;
    int n_out;               // n_pairs * K
    const int* pairs;        // [n_pairs] (only read when y_obs != nullptr)
    const float2* y_obs;     // full measurement vector [P*K] or nullptr
    const unsigned char* fmask;  // [K]: rows with fmask[k] == 0 get a zero residual (nullptr = all rows)
    float2* out;             // [n_pairs * K]
    long long partial_elems = 0;   // extent of partial (checked in the bounds-checked build)
};

struct AdjArgs {
    const int* pairs;        // [n_pairs]
    int n_pairs;
    const float2* r;         // [n_pairs * K]
    float2* g_out;           // [N] plain adjoint output, or nullptr
    float2* s;               // [N] SPGM iterate updated in place, or nullptr
    float step;              // eta / B
    float alpha;             // eta * lambda * w1 (soft-threshold level)
    float shrink;            // 1 / (1 + eta * lambda * w2) (elastic-net scaling; 1 for plain l1)
    float alpha_g = 0.f;     // eta * lambda * w3: group shrink over 2 x 2 x 1 voxel blocks (expansion adjoints; 0 = off)
    int pchunk;              // pairs staged in shared memory per round
    long long r_elems = 0;   // extent of r (checked in the bounds-checked build)
};

// per (antenna, tile) FP64 set-up
struct AntSetup {
    const double* ant_xyz;   // [(T+R)][3]
    int n_ant;
    double x0, y0, z0, dx, dy, dz;
    double f0c, dfc, dfc2;   // f0/c, df/c, K2 df/c
    AntTile* out;            // [n_ant * n_tiles]
    const double* tile_c = nullptr;    // explicit voxel positions: tile centres [n_tiles][3] (FP64)
    const double* vox_xyz = nullptr;   //                           voxel positions [n_vox][3] (FP64)
    long long n_vox = 0;
};

constexpr int GEN_MAX_K = 128;    // frequencies of the general-frequency path
constexpr int GEN_ADJ_PCHUNK = 16;
// Arbitrary frequency lists: per-(antenna, tile, k) reduced phases and f_k / c (hi + lo).
struct GenDesc {
    const float* antk;       // [(T + R) * n_tiles * K]
    const float2* fkc;       // [K]
};
cudaError_t launch_antk_setup(const GridDesc& g, const AntSetup& a, const double* fk_over_c, int K, float* out,
                              cudaStream_t st);
cudaError_t launch_fwd_general(const OpDesc& op, const GenDesc& gd, const FwdArgs& a, dim3 grid, cudaStream_t st);
cudaError_t launch_adj_general(const OpDesc& op, const GenDesc& gd, const AdjArgs& a, cudaStream_t st);
const void* fwd_general_ptr();

// Chebyshev-expansion operator (op_cheb.cu)
constexpr int CHEB_THREADS = 128;
constexpr int CHEB_GROUP = 4;                              // lanes per (pair, tile) in the forward
constexpr int CHEB_GROUPS = CHEB_THREADS / CHEB_GROUP;    // 32
constexpr int CHEB_ADJ_PCHUNK = 16;                        // pairs staged per adjoint round (128-voxel tiles)
// pairs staged per round of the expansion adjoint over blocks of 8 x 4 x tz voxels (tz = TILE_Z: the tiles;
// tz = 2 TILE_Z: two tiles along z, 256 threads)
__host__ __device__ constexpr int adj_cheb_pchunk(int tz) { return tz == TILE_Z ? CHEB_ADJ_PCHUNK : 2 * CHEB_ADJ_PCHUNK; }
constexpr int CHEB_MIN_L = 10;
constexpr int CHEB_MAX_L = 32;
struct ChebDesc {
    const float* coef;       // [k_pad][round4(L)] b_l(z_k), z_k = (k - k_c) z_step; zero for k >= K or l >= L
    float tau;               // t = tau * delta
    int L;                   // expansion terms (even, 10 ... 32)
    int k_pad;               // K rounded up to a multiple of 4
    float fc_hi, fc_lo;      // f_c / c (cycles per metre) as hi + lo, f_c = f_0 + k_c df the band centre
};
// Shared-memory row stride (floats) of the forward's coefficient table: round4(L), plus 4 where that is a
// multiple of 16, so that the 4 rows a lane group reads at once start in different banks.
__host__ __device__ constexpr int fwd_coef_stride(int LT)
{
    return ((LT + 3) & ~3) % 16 == 0 ? ((LT + 3) & ~3) + 4 : ((LT + 3) & ~3);
}
// Rows of the coefficient table the forward holds in shared memory: k <= K/2 (k_pad = K rounded up to 4), the
// rows the mirror-folded expansion reads (k < K/2 and, for odd K, the centre row).
__host__ __device__ constexpr int fwd_coef_rows(int k_pad) { return k_pad / 2 + 1; }
// points: the geometry has explicit voxel positions (per-stage voxel offsets are staged too)
size_t fwd_cheb_smem_bytes(int LT, int k_pad, int pch, int threads, int group, bool points = false,
                           int tz = TILE_Z);
size_t adj_cheb_smem_bytes(int LT, int k_pad, int tz = TILE_Z);
const void* fwd_cheb_kernel_ptr(int LT, int group, int tz = TILE_Z);   // nullptr where not built
const void* adj_cheb_kernel_ptr(int LT, int tz = TILE_Z);   // nullptr where not built (tz = 8: L <= 24)
// threads: 64 or 128; group: 4 or 8 lanes per (pair, tile); a.VS = pairs per CTA, a power of two
// dividing threads / group
cudaError_t launch_fwd_cheb(const OpDesc& op, const ChebDesc& cd, const FwdArgs& a, dim3 grid, int threads,
                            int group, int tz, size_t smem, cudaStream_t st);
cudaError_t launch_adj_cheb(const OpDesc& op, const ChebDesc& cd, const AdjArgs& a, int tz, size_t smem,
                            cudaStream_t st);
// tensor-core (tcgen05) expansion stage of the forward (op_cheb_tc_fwd.cu): 256 threads, a.VS = pairs per
// CTA in {16, 32, 64}, K <= 128
size_t fwd_cheb_tc_smem_bytes(int LT, int K, int pch);
const void* fwd_cheb_tc_kernel_ptr(int LT, bool f16);
cudaError_t launch_fwd_cheb_tc(const OpDesc& op, const ChebDesc& cd, const FwdArgs& a, dim3 grid, bool f16,
                               size_t smem, cudaStream_t st);
// tensor-core (tcgen05) coefficient stage of the expansion adjoint (op_cheb_tc.cu), K <= 128, L <= 32
size_t adj_cheb_tc_smem_bytes(int K, int L);
const void* adj_cheb_tc_kernel_ptr(int LT, bool f16);
cudaError_t launch_adj_cheb_tc(const OpDesc& op, const ChebDesc& cd, const AdjArgs& a, bool f16, size_t smem,
                               cudaStream_t st);

// One launch over the same phase of several scenes (batched SPGM): item i covers the CTAs
// [cta0_i, cta0_{i+1}) of the launch; the items of a launch are sorted by cta0, the first at 0.
struct MultiFwdItem {
    OpDesc op;
    ChebDesc cd;             // coefficient table padded to the launch's expansion length (zero rows beyond L)
    FwdArgs a;
    int n_groups;            // pair groups of the scene (CTA = pair group + n_groups * chunk)
    int cta0;
};
struct MultiRedItem {
    OpDesc op;
    ReduceArgs a;
    int cta0;
};
struct MultiAdjItem {
    OpDesc op;
    ChebDesc cd;
    AdjArgs a;
    int cta0;                // CTA = voxel tile of the scene
};
cudaError_t launch_fwd_cheb_multi(int LT, const MultiFwdItem* items, int n_items, int n_ctas, size_t smem,
                                  cudaStream_t st);
cudaError_t launch_adj_cheb_multi(int LT, const MultiAdjItem* items, int n_items, int n_ctas, size_t smem,
                                  cudaStream_t st);
cudaError_t launch_fwd_reduce_multi(const MultiRedItem* items, int n_items, int n_ctas, cudaStream_t st);
const void* fwd_cheb_multi_ptr(int LT);
const void* adj_cheb_multi_ptr(int LT);
int fwd_reduce_blocks(int n_out);

constexpr int FWD_PC = 8;         // pairs per forward CTA
constexpr int ADJ_TC_PCHUNK = 8;  // pairs whose tensor-core B operands a CTA holds at once
constexpr int ADJ_THREADS = 128;  // one 8x4x4 tile: two voxels per thread, pairs split in two halves
constexpr int ADJ_PCHUNK = 32;

size_t fwd_smem_bytes(int K1, int nt);

// Launch with programmatic stream serialisation (the kernel may start while the
// previous kernel in the stream finishes; it calls pdl_wait() before reading
// that kernel's results).
inline cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void** args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}
const void* fwd_kernel_ptr(int K1);
const void* adj_kernel_ptr(int K1);
size_t adj_smem_bytes(int K1, int pchunk);

cudaError_t launch_fwd_partial(const OpDesc& op, const FwdArgs& a, dim3 grid, int nt, size_t smem,
                               cudaStream_t st);
cudaError_t launch_fwd_reduce(const OpDesc& op, const ReduceArgs& a, cudaStream_t st);
cudaError_t launch_adjoint(const OpDesc& op, const AdjArgs& a, size_t smem, cudaStream_t st);
// tensor-core adjoint: prep kernel (B operands of every pair into bmat) + tcgen05 kernel
size_t adj_tc_smem_bytes(int pchunk);
size_t adj_tc_bmat_bytes(int n_pairs);
const void* adj_tc_kernel_ptr(int K1, bool f16);
cudaError_t launch_adjoint_tc(const OpDesc& op, const AdjArgs& a, bool f16, const float2* r, unsigned char* bmat,
                              float* inv_scale, size_t smem, cudaStream_t st);
cudaError_t launch_ant_setup(const GridDesc& g, const AntSetup& a, cudaStream_t st);
// FP64 max over antennas, tiles and voxel slots of | |r_a - r_v| - |r_a - r_c| | (atomicMax on the bits)
cudaError_t launch_cheb_range(const GridDesc& g, const AntSetup& a, unsigned long long* out, cudaStream_t st);

// FP64 reductions (deterministic: fixed grid, fixed tree)
constexpr int RED_BLOCKS = 256;
cudaError_t launch_norm2(const float2* v, long long n, double* partial, double* out, cudaStream_t st);
cudaError_t launch_abs_sum(const float2* v, long long n, double* partial, double* out, cudaStream_t st);
cudaError_t launch_abs_max(const float2* v, long long n, double* partial, double* out, cudaStream_t st);
// out = max_n | |a_n| - |b_n| |  (FP64)
cudaError_t launch_mag_change(const float2* a, const float2* b, long long n, double* partial, double* out,
                              cudaStream_t st);
// out = shrink prox_alpha(s - step g)  and its backward (grad_s, grad_g may be null; out3[0] = dL/dstep,
// out3[1] = dL/dalpha, out3[2] = dL/dshrink in FP64; partial holds 3*RED_BLOCKS doubles)
cudaError_t launch_prox_step(const float2* s, const float2* g, float step, float alpha, float shrink, long long n,
                             float2* out, cudaStream_t st);
cudaError_t launch_prox_step_backward(const float2* s, const float2* g, float step, float alpha, float shrink,
                                      long long n, const float2* go, float2* grad_s, float2* grad_g, double* partial,
                                      double* out3, cudaStream_t st);
// out = shrink G_alpha_g(prox_alpha(s - step g)) with the block shrink G over the 2 x 2 x 1 voxel blocks of an
// nx x ny x nz grid, and its backward (out4 = dL/dstep, dL/dalpha, dL/dalpha_g, dL/dshrink in FP64; partial
// holds 4*RED_BLOCKS doubles)
cudaError_t launch_prox_group_step(const float2* s, const float2* g, float step, float alpha, float alpha_g,
                                   float shrink, int nx, int ny, int nz, float2* out, cudaStream_t st);
cudaError_t launch_prox_group_step_backward(const float2* s, const float2* g, float step, float alpha, float alpha_g,
                                            float shrink, int nx, int ny, int nz, const float2* go, float2* grad_s,
                                            float2* grad_g, double* partial, double* out4, cudaStream_t st);
// out = sum over the 2 x 2 x 1 voxel blocks (ix/2, iy/2, iz) of the block's l2 norm (FP64, fixed tree)
cudaError_t launch_group_norm_sum(const float2* v, int nx, int ny, int nz, double* partial, double* out,
                                  cudaStream_t st);
// dst = src / sqrt(*nrm2)
cudaError_t launch_normalize(const float2* src, float2* dst, long long n, const double* nrm2, cudaStream_t st);
// out[0] = a[0] / (scale * b[0])
cudaError_t launch_ratio(const double* a, const double* b, double scale, double* out, cudaStream_t st);
// out[0] = a[0] * sa + b[0] * sb
cudaError_t launch_axpby(const double* a, double sa, const double* b, double sb, double* out, cudaStream_t st);

}  // namespace nfm
