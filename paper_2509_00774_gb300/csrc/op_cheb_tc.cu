// Tensor-core (tcgen05) form of the Chebyshev-expansion adjoint (the precision
// modes NFM_TC_BF16X3 / NFM_TC_FP16X3 for equally spaced frequencies).
//
// The expansion adjoint (op_cheb.cu) needs, per (pair j, tile t), the
// coefficients
//
//     C_l = j^l sum_k b_l(k) r'_k,   r'_k = conj(p_k) r_jk e^{+j 2 pi k df D_c(j, t)/c},
//
// a dense contraction over the K frequencies with a real, constant b.  For four
// tiles and a chunk of 16 pairs it is one real GEMM D = A B^T:
//
//     A[(t, j, c), k] = Re / Im r'_k (c = 0 / 1)   M = 128 rows (4 tiles x 16 pairs x 2)
//     B[l, k]         = b_l(k)                     N = 32 (l < L, zero rows above)
//     D[(t, j, c), l] = sum_k A B                  K = the frequencies (multiple of 16, zero padded)
//
// Both operands are split x = hi + lo in BF16 (or FP16, r' scaled per pair by a
// power of two) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in FP32 in
// tensor memory (3 tcgen05.mma of M128 N32 K16 per K step, one thread issues,
// completion through tcgen05.commit -> mbarrier with a bounded wait).  A is built
// and multiplied in two parts of the K range through one buffer, so that the
// shared memory of two CTAs fits on an SM (the other CTA's per-voxel work covers
// each part's wait).  Warps 0-3
// read D back (lane = row) into shared memory; the per-voxel part, sum_l T_l(t)
// C_l with the Chebyshev recurrence and the fused step/prox epilogue, stays on
// the CUDA cores exactly as in the FP32 expansion adjoint.
//
// CTA = 4 tiles = 512 threads (thread = voxel).  Operands use the no-swizzle
// K-major layout of tc_ptx.cuh.
#include "nfm_kernels.cuh"
#include "cheb_device.cuh"
#include "tc_ptx.cuh"

namespace nfm {

namespace {

using namespace tc;

constexpr int CTC_TILES = 4;                       // tiles per CTA
constexpr int CTC_THREADS = CTC_TILES * TILE_V;    // 512
constexpr int CTC_PCH = 16;                        // pairs per chunk
constexpr int CTC_M = CTC_TILES * CTC_PCH * 2;     // 128 rows (tile, pair, re/im)
constexpr int CTC_N = 32;                          // l, L <= 32
constexpr int CTC_KSTEP_A = CTC_M * 16 * 2;        // 4096 bytes: one K step of A
constexpr int CTC_KSTEP_B = CTC_N * 16 * 2;        // 1024 bytes: one K step of B
constexpr int CTC_CRS = CTC_N + 2;                 // float2 row stride of the read-back D (16-byte rows,
                                                   // two rows per bank group: 2-way stores, not 16-way)

template <bool F16>
__host__ __device__ constexpr uint32_t ctc_idesc()
{
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(CTC_N >> 3) << 17) |
           ((uint32_t)(CTC_M >> 4) << 24);
}

struct CtcSmem {   // K-step counts and byte offsets of the dynamic shared-memory regions
    int ks, nh, ksp;   // K steps (zero-padded to whole parts), parts of the K range, K steps per part
    int a, b, pt, p8, craw, rbuf, scale, bar, tslot, total;
    __host__ __device__ explicit CtcSmem(int K)
    {
        const int ks0 = (K + 15) / 16;
        nh = ks0 >= 2 ? 2 : 1;
        ksp = (ks0 + nh - 1) / nh;
        ks = nh * ksp;
        const int KS = ks;
        a = 0;                                            // [split 2][ksp][4096]: one part of A
        b = a + 2 * ksp * CTC_KSTEP_A;                    // [split 2][KS][1024]
        pt = b + 2 * KS * CTC_KSTEP_B;                    // [4 tiles][16 pairs] PairTile
        p8 = pt + CTC_TILES * CTC_PCH * (int)sizeof(PairTile);     // [4][16] float2 e^{+j 2 pi 8 df D_c/c}
        craw = p8 + CTC_TILES * CTC_PCH * (int)sizeof(float2);     // [4][16][CTC_CRS] float2 (D_re, D_im)
        rbuf = craw + CTC_TILES * CTC_PCH * CTC_CRS * (int)sizeof(float2);    // [16 pairs][16 KS + 1] float2 r
        scale = rbuf + CTC_PCH * (16 * KS + 1) * (int)sizeof(float2);     // [16] float
        bar = scale + CTC_PCH * (int)sizeof(float);       // one mbarrier (8-byte aligned)
        tslot = bar + 8;
        total = tslot + 16;
    }
};

}  // namespace

template <int LT, bool F16>
__global__ void __launch_bounds__(CTC_THREADS, 2) adj_cheb_tc_kernel(OpDesc op, ChebDesc cd, AdjArgs a)
{
    constexpr int LS = (LT + 3) & ~3;        // table row stride of the coefficient table
    extern __shared__ __align__(1024) unsigned char smem[];
    const int K = op.K;
    const CtcSmem L(K);
    const int KS = L.ks, KSP = L.ksp, NH = L.nh;
    unsigned char* As = smem + L.a;
    unsigned char* Bs = smem + L.b;
    PairTile* pt = reinterpret_cast<PairTile*>(smem + L.pt);
    float2* p8 = reinterpret_cast<float2*>(smem + L.p8);
    float2* craw = reinterpret_cast<float2*>(smem + L.craw);
    float2* rbuf = reinterpret_cast<float2*>(smem + L.rbuf);
    const int RB = 16 * KS + 1;              // rbuf row stride (odd: the 8 rows a warp reads use distinct banks)
    float* scale = reinterpret_cast<float*>(smem + L.scale);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);

    const int tid = threadIdx.x;
    const int warp = tid / 32;
    const int t4 = tid / TILE_V;             // tile of this thread within the CTA
    const int v = tid % TILE_V;              // voxel within the tile
    const int tile = blockIdx.x * CTC_TILES + t4;
    const bool tile_ok = tile < op.g.n_tiles;
    int tx = 0, ty = 0, tz = 0;
    if (tile_ok) tile_coords(op.g, tile, tx, ty, tz);
    const int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y);
    const VoxelOffset o = voxel_offset(op.g, lx, ly, lz);
    constexpr uint32_t IDESC = ctc_idesc<F16>();

    if (warp == 0) {
        tmem_alloc(tslot, 32);
        tmem_relinquish();
    }
    if (tid == 0) mbar_init(bar, 1);
    // B = the coefficient table b_l(k), rows l (zero for l >= LT), two k per 32-bit word.  A row's
    // words sit in 4 banks of the K-major layout, so the lanes of a warp take 8 rows x 4 words.
    for (int e = tid; e < CTC_N * KS * 8; e += CTC_THREADS) {
        const int eh = e >> 5;
        const int l = (eh / (KS * 2)) * 8 + ((e >> 2) & 7);
        const int kp = (eh % (KS * 2)) * 4 + (e & 3);
        const int k = 2 * kp;
        const float b0 = (l < LT && k < K) ? cd.coef[k * LS + l] : 0.f;
        const float b1 = (l < LT && k + 1 < K) ? cd.coef[(k + 1) * LS + l] : 0.f;
        uint32_t hi, lo;
        split2<F16>(b0, b1, hi, lo);
        const int s = k / 16, kk = k % 16;
        *reinterpret_cast<uint32_t*>(Bs + 0 * KS * CTC_KSTEP_B + s * CTC_KSTEP_B + kmaj_off(l, kk)) = hi;
        *reinterpret_cast<uint32_t*>(Bs + 1 * KS * CTC_KSTEP_B + s * CTC_KSTEP_B + kmaj_off(l, kk)) = lo;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    bool ok = true, hold = false;
    uint32_t n_waits = 0;                    // completed commit -> mbarrier phases
    float gr = 0.f, gi = 0.f;

    for (int c0 = 0; c0 < a.n_pairs; c0 += CTC_PCH) {
        const int nc = min(CTC_PCH, a.n_pairs - c0);
        // pair tiles of the chunk (geometry only: no kernel of this library writes it)
        if (tid < CTC_TILES * CTC_PCH) {
            const int tt = tid / CTC_PCH, j = tid % CTC_PCH;
            const int til = blockIdx.x * CTC_TILES + tt;
            if (j < nc && til < op.g.n_tiles) {
                pt[tid] = load_pair_tile(op, a.pairs[c0 + j], til);
                p8[tid] = tile_step_cis_exact(pt[tid], 8);
            }
        }
        if (c0 == 0) {
            pdl_wait();                      // r comes from the previous kernel
            // a tensor-core forward of the same step whose wait ran out left r stale: keep the iterate
            hold = (*reinterpret_cast<volatile int*>(op.err) & ERRF_TIMEOUT) != 0;
        }
        // the chunk's residual rows into shared memory (all copies in flight at once)
        for (int e = tid; e < nc * K; e += CTC_THREADS) {
            const int j = e / K, k = e - j * K;
            cp_async_8(rbuf + j * RB + k, a.r + (size_t)c0 * K + e, true);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        // FP16: per-pair power-of-two scale so that |Re r'|, |Im r'| <= |r'| < 1
        if (F16) {
            for (int j = warp; j < CTC_PCH; j += CTC_THREADS / 32) {
                float m = 0.f;
                if (j < nc)
                    for (int k = tid % 32; k < K; k += 32) {
                        float2 r = rbuf[j * RB + k];
                        if (op.pulse) r = cmul_conj(r, op.pulse[k]);
                        m = fmaxf(m, sqrtf(r.x * r.x + r.y * r.y));   // |r'| = |conj(p) r|
                    }
                for (int w = 16; w > 0; w >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, w));
                if (tid % 32 == 0) {
                    float sc = 1.0f;
                    if (m > 0.f) {
                        int ex;
                        frexpf(m, &ex);
                        sc = ldexpf(1.0f, -ex);
                    }
                    scale[j] = sc;
                }
            }
            __syncthreads();
        }
        // A = r' rows (tile, pair, re/im), two k per 32-bit word, one part of the K range (KSP K steps) at a
        // time.  Thread: row tj = 8 (warp % 8) + lane / 4 and word w4 = lane % 4 of the part's k-pairs
        // kp = 4 KSP (warp / 8) + 4 m + w4, m < KSP; a warp stores 8 rows x 4 words at a time (distinct banks
        // in the K-major layout), and the phasors of k and k + 1 advance by the exact 8-step phasor from one
        // SFU start each.  The part's MMAs are committed and waited for before the next part is written.
        const bool issue = !(op.hooks & HOOK_TC_SKIP_ISSUE);
        for (int part = 0; part < NH; ++part) {
            const int w4 = tid & 3, tj = ((warp & 7) << 3) + ((tid >> 2) & 7), h = warp >> 3;
            const int tt = tj / CTC_PCH, j = tj % CTC_PCH;
            const bool valid = j < nc && blockIdx.x * CTC_TILES + tt < op.g.n_tiles;
            const int kp0 = part * 8 * KSP + h * 4 * KSP + w4;       // global k-pair index of m = 0
            float2 c0v = make_float2(0.f, 0.f), c1v = c0v, W8 = c0v;
            float sc = 1.0f;
            if (valid) {
                const PairTile& P = pt[tj];
                c0v = tile_step_cis(P, 2 * kp0);
                c1v = tile_step_cis(P, 2 * kp0 + 1);
                W8 = p8[tj];
                if (F16) sc = scale[j];
            }
            const float2* rr = rbuf + j * RB;
            // byte offsets of the re / im rows' words at m = 0 within the part's A buffer: the word of
            // local k = 8 q + 2 w4 sits in K step q / 2, 8-column half q % 2 (q = (k_local >> 3))
            const uint32_t row_re = kmaj_off(2 * tj, 2 * w4), row_im = kmaj_off(2 * tj + 1, 2 * w4);
            const int q0 = h * KSP;                                   // (2 kp0 - part * 16 KSP) >> 3
            for (int m = 0; m < KSP; ++m) {
                const int k = 2 * (kp0 + 4 * m);
                float2 v0 = make_float2(0.f, 0.f), v1 = v0;
                if (valid) {
                    if (k < K) {
                        float2 r = rr[k];
                        if (op.pulse) r = cmul_conj(r, op.pulse[k]);
                        v0 = cmul(r, c0v);
                        if (F16) {
                            v0.x *= sc;
                            v0.y *= sc;
                        }
                    }
                    if (k + 1 < K) {
                        float2 r = rr[k + 1];
                        if (op.pulse) r = cmul_conj(r, op.pulse[k + 1]);
                        v1 = cmul(r, c1v);
                        if (F16) {
                            v1.x *= sc;
                            v1.y *= sc;
                        }
                    }
                    c0v = cmul(c0v, W8);
                    c1v = cmul(c1v, W8);
                }
                uint32_t hre, lre, him, lim;
                split2<F16>(v0.x, v1.x, hre, lre);
                split2<F16>(v0.y, v1.y, him, lim);
                const int q = q0 + m;
                unsigned char* a0 = As + (q >> 1) * CTC_KSTEP_A + (q & 1) * 128;
                *reinterpret_cast<uint32_t*>(a0 + row_re) = hre;
                *reinterpret_cast<uint32_t*>(a0 + row_im) = him;
                *reinterpret_cast<uint32_t*>(a0 + KSP * CTC_KSTEP_A + row_re) = lre;
                *reinterpret_cast<uint32_t*>(a0 + KSP * CTC_KSTEP_A + row_im) = lim;
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0 && issue) {
                tc_fence_after();
                const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
                for (int sl = 0; sl < KSP; ++sl) {
                    const int sg = part * KSP + sl;                    // K step of B
                    const uint64_t ahi = smem_desc(a_base + sl * CTC_KSTEP_A);
                    const uint64_t alo = smem_desc(a_base + (KSP + sl) * CTC_KSTEP_A);
                    const uint64_t bhi = smem_desc(b_base + sg * CTC_KSTEP_B);
                    const uint64_t blo = smem_desc(b_base + (KS + sg) * CTC_KSTEP_B);
                    tc_mma(tbase, ahi, bhi, IDESC, (part > 0 || sl > 0) ? 1u : 0u);
                    tc_mma(tbase, ahi, blo, IDESC, 1u);
                    tc_mma(tbase, alo, bhi, IDESC, 1u);
                }
                tc_commit(bar);
            }
            // the wait's outcome is made uniform over the CTA: on a timeout no thread reads TMEM, no further
            // MMA is issued and the iterate (or g) is left unwritten; the MMAs already committed get one more
            // bounded wait so that none is in flight when TMEM is released
            if (!__syncthreads_and(mbar_wait(bar, n_waits & 1u, op.wait_ns))) {
                if (issue) mbar_wait(bar, n_waits & 1u, op.wait_ns);
                ok = false;
                break;
            }
            ++n_waits;
        }
        if (!ok) break;
        tc_fence_after();
        if (warp < 4) {                      // lanes 32 warp .. : rows (tile, pair, re/im)
            float d[32];
            tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16), d);
            const int row = tid;             // tid < 128
            const int tt = row / (2 * CTC_PCH), j = (row / 2) % CTC_PCH, c = row & 1;
            const float inv = F16 ? 1.0f / scale[j] : 1.0f;
            float* dst = reinterpret_cast<float*>(craw + (tt * CTC_PCH + j) * CTC_CRS) + c;
#pragma unroll
            for (int l = 0; l < CTC_N; ++l) dst[2 * l] = d[l] * inv;
        }
        tc_fence_before();
        __syncthreads();
        // per voxel: sum over the chunk's pairs of conj(u') sum_l T_l(t) j^l (D_re + j D_im)_l
        if (tile_ok) {
            for (int j = 0; j < nc; ++j) {
                const ChebVoxel cv = cheb_voxel(pt[t4 * CTC_PCH + j], o, cd.fc_hi, cd.fc_lo);
                const float2 c0v = cis_turns_sfu(cv.th0);
                const float t = cv.delta * cd.tau, t2 = t + t;
                const float4* C = reinterpret_cast<const float4*>(craw + (t4 * CTC_PCH + j) * CTC_CRS);
                float4 q = C[0];                 // (D_0, D_1): factors 1 and j
                float ar = fmaf(t, -q.w, q.x), ai = fmaf(t, q.z, q.y);
                float Tp = 1.f, Tc = t;
#pragma unroll
                for (int l = 2; l < LT; l += 2) {
                    q = C[l / 2];                // (D_l, D_l+1)
                    const float Ta = fmaf(t2, Tc, -Tp);
                    const float Tb = fmaf(t2, Ta, -Tc);
                    if ((l & 3) == 0) {          // factors 1 and j
                        ar = fmaf(Ta, q.x, ar);
                        ai = fmaf(Ta, q.y, ai);
                        ar = fmaf(Tb, -q.w, ar);
                        ai = fmaf(Tb, q.z, ai);
                    } else {                     // factors -1 and -j
                        ar = fmaf(Ta, -q.x, ar);
                        ai = fmaf(Ta, -q.y, ai);
                        ar = fmaf(Tb, q.w, ar);
                        ai = fmaf(Tb, -q.z, ai);
                    }
                    Tp = Ta;
                    Tc = Tb;
                }
                const float wr = cv.amp * c0v.x, wi = cv.amp * c0v.y;
                gr = fmaf(wr, ar, fmaf(-wi, ai, gr));
                gi = fmaf(wr, ai, fmaf(wi, ar, gi));
            }
        }
        __syncthreads();                     // craw, pt and A are rewritten by the next chunk
    }
    pdl_launch_dependents();
    if (!ok && tid == 0) atomicOr(op.err, ERRF_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 32);
    }

    if (!tile_ok || !ok || (hold && a.s)) return;   // uniform over a warp (a warp lies in one tile; ok per CTA)
    const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
    const bool in_grid = ix < op.g.nx && iy < op.g.ny && iz < op.g.nz;
    const size_t n = in_grid ? ((size_t)iz * op.g.ny + iy) * op.g.nx + ix : 0;
    if (a.s) {                               // every lane of the warp takes part (group norms)
        const float2 sv = in_grid ? a.s[n] : make_float2(0.f, 0.f);
        const float2 out = step_prox(sv, gr, gi, a.step, a.alpha, a.alpha_g, a.shrink, in_grid);
        if (in_grid) a.s[n] = out;
    } else if (in_grid) {
        a.g_out[n] = make_float2(gr, gi);
    }
}

size_t adj_cheb_tc_smem_bytes(int K)
{
    return (size_t)CtcSmem(K).total;
}

template <bool F16>
static const void* adj_cheb_tc_ptr_f(int LT)
{
    switch (LT) {
    case 10: return (const void*)adj_cheb_tc_kernel<10, F16>;
    case 12: return (const void*)adj_cheb_tc_kernel<12, F16>;
    case 14: return (const void*)adj_cheb_tc_kernel<14, F16>;
    case 16: return (const void*)adj_cheb_tc_kernel<16, F16>;
    case 18: return (const void*)adj_cheb_tc_kernel<18, F16>;
    case 20: return (const void*)adj_cheb_tc_kernel<20, F16>;
    case 22: return (const void*)adj_cheb_tc_kernel<22, F16>;
    case 24: return (const void*)adj_cheb_tc_kernel<24, F16>;
    case 26: return (const void*)adj_cheb_tc_kernel<26, F16>;
    case 28: return (const void*)adj_cheb_tc_kernel<28, F16>;
    case 30: return (const void*)adj_cheb_tc_kernel<30, F16>;
    case 32: return (const void*)adj_cheb_tc_kernel<32, F16>;
    default: return nullptr;
    }
}

const void* adj_cheb_tc_kernel_ptr(int LT, bool f16)
{
    return f16 ? adj_cheb_tc_ptr_f<true>(LT) : adj_cheb_tc_ptr_f<false>(LT);
}

cudaError_t launch_adj_cheb_tc(const OpDesc& op, const ChebDesc& cd, const AdjArgs& a, bool f16, size_t smem,
                               cudaStream_t st)
{
    const void* fn = adj_cheb_tc_kernel_ptr(cd.L, f16);
    if (!fn || op.K > GEN_MAX_K || cd.L > CTC_N) return cudaErrorInvalidValue;
    void* args[] = {(void*)&op, (void*)&cd, (void*)&a};
    const unsigned grid = (unsigned)((op.g.n_tiles + CTC_TILES - 1) / CTC_TILES);
    return launch_pdl(fn, dim3(grid), dim3(CTC_THREADS), smem, st, args);
}

}  // namespace nfm
