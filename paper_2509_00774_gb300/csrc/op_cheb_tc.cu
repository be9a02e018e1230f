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
// completion through tcgen05.commit -> mbarrier with a bounded wait).  The MMAs
// of one chunk run while the CTA does the per-voxel work of the previous chunk, so
// the wait normally finds them done.  Warps 0-3
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
template <bool F16>
__host__ __device__ constexpr uint32_t ctc_idesc()
{
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(CTC_N >> 3) << 17) |
           ((uint32_t)(CTC_M >> 4) << 24);
}

struct CtcSmem {   // K steps and byte offsets of the dynamic shared-memory regions
    int ks;
    int a, b, pt, p8, craw, rbuf, scale, bar, tslot, total;
    __host__ __device__ CtcSmem(int K, int LT)
    {
        ks = (K + 15) / 16;
        const int KS = ks;
        a = 0;                                                      // [split 2][KS][4096]
        b = a + 2 * KS * CTC_KSTEP_A;                               // [split 2][KS][1024]
        pt = b + 2 * KS * CTC_KSTEP_B;                              // [2 chunks][4 tiles][16 pairs] PairTile
        p8 = pt + 2 * CTC_TILES * CTC_PCH * (int)sizeof(PairTile);  // [2][4][16] float2 e^{+j 2 pi 8 df D_c/c}
        craw = p8 + 2 * CTC_TILES * CTC_PCH * (int)sizeof(float2);  // [4][16][LT] float2 C_l
        rbuf = craw + CTC_TILES * CTC_PCH * LT * (int)sizeof(float2);         // [16 pairs][16 KS + 8] float2 r
        scale = rbuf + CTC_PCH * (16 * KS + 8) * (int)sizeof(float2);         // [16] float
        bar = scale + CTC_PCH * (int)sizeof(float);                 // one mbarrier (8-byte aligned)
        tslot = bar + 8;
        total = tslot + 16;
    }
};

}  // namespace

// Chunks of 16 pairs are software-pipelined: iteration c builds A for chunk c and issues its MMAs, then
// runs the per-voxel sum of chunk c - 1 (whose coefficients were read back in iteration c - 1) while
// the tensor core works, then waits, reads chunk c's coefficients back and stages chunk c + 1 (pair
// tiles into the other buffer; r, already in flight since the MMAs were issued).
template <int LT, bool F16>
__global__ void __launch_bounds__(CTC_THREADS, 2) adj_cheb_tc_kernel(OpDesc op, ChebDesc cd, AdjArgs a)
{
    constexpr int LS = (LT + 3) & ~3;        // table row stride of the coefficient table
    constexpr int CRS = LT;                  // float2 row stride of the read-back coefficients (16-byte rows)
    extern __shared__ __align__(1024) unsigned char smem[];
    const int K = op.K;
    const CtcSmem L(K, LT);
    const int KS = L.ks;
    unsigned char* As = smem + L.a;
    unsigned char* Bs = smem + L.b;
    PairTile* pt_s = reinterpret_cast<PairTile*>(smem + L.pt);
    float2* p8_s = reinterpret_cast<float2*>(smem + L.p8);
    float2* craw = reinterpret_cast<float2*>(smem + L.craw);
    float2* rbuf = reinterpret_cast<float2*>(smem + L.rbuf);
    // rbuf row stride: 16-byte rows, and 16 words mod 32 so that the two rows x four k-pairs of a
    // quarter warp's 16-byte loads fall in distinct banks
    const int RB = 16 * KS + 8;
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
    const bool issue = !(op.hooks & HOOK_TC_SKIP_ISSUE);
    const int n_chunks = (a.n_pairs + CTC_PCH - 1) / CTC_PCH;

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

    // pair tiles of chunk c into buffer c & 1 (geometry only: no kernel of this library writes it)
    auto load_tiles = [&](int c) {
        if (tid < CTC_TILES * CTC_PCH) {
            const int c0 = c * CTC_PCH, nc = min(CTC_PCH, a.n_pairs - c0);
            const int tt = tid / CTC_PCH, j = tid % CTC_PCH;
            const int til = blockIdx.x * CTC_TILES + tt;
            if (j < nc && til < op.g.n_tiles) {
                PairTile* P = pt_s + (c & 1) * CTC_TILES * CTC_PCH;
                P[tid] = load_pair_tile(op, a.pairs[c0 + j], til);
                p8_s[(c & 1) * CTC_TILES * CTC_PCH + tid] = tile_step_cis_exact(P[tid], 8);
            }
        }
    };
    // the residual rows of chunk c into rbuf (all copies in flight at once, one commit group)
    auto load_r = [&](int c) {
        const int c0 = c * CTC_PCH, nc = min(CTC_PCH, a.n_pairs - c0);
        for (int e = tid; e < nc * K; e += CTC_THREADS) {
            const int j = e / K, k = e - j * K;
            cp_async_8(rbuf + j * RB + k, a.r + NFM_IDX((long long)c0 * K + e, a.r_elems, op.err), true);
        }
        cp_async_commit();
    };
    float gr = 0.f, gi = 0.f;
    // per voxel: sum over chunk c's pairs of conj(u') sum_l T_l(t) j^l (D_re + j D_im)_l
    auto voxel_sum = [&](int c) {
        if (!tile_ok) return;
        const int nc = min(CTC_PCH, a.n_pairs - c * CTC_PCH);
        const PairTile* P = pt_s + (c & 1) * CTC_TILES * CTC_PCH + t4 * CTC_PCH;
        for (int j = 0; j < nc; ++j) {
            const ChebVoxel cv = cheb_voxel(P[j], o, cd.fc_hi, cd.fc_lo);
            const float2 c0v = cis_turns_sfu(cv.th0);
            const float t = cv.delta * cd.tau, t2 = t + t;
            const float4* C = reinterpret_cast<const float4*>(craw + (t4 * CTC_PCH + j) * CRS);
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
    };

    if (n_chunks > 0) load_tiles(0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    bool ok = true;
    uint32_t n_waits = 0;                    // completed commit -> mbarrier phases
    pdl_wait();                              // r comes from the previous kernel
    // a tensor-core forward of the same step whose wait ran out left r stale: keep the iterate
    const bool hold = (*reinterpret_cast<volatile int*>(op.err) & ERRF_TIMEOUT) != 0;
    if (n_chunks > 0) load_r(0);
    cp_async_wait_all();
    __syncthreads();

    for (int c = 0; c < n_chunks; ++c) {
        const int c0 = c * CTC_PCH, nc = min(CTC_PCH, a.n_pairs - c0);
        const int buf = (c & 1) * CTC_TILES * CTC_PCH;
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
        // A = r' rows (tile, pair, re/im), two k per 32-bit word.  Thread: row tj = 8 (warp % 8) +
        // lane / 4 and word w4 = lane % 4 of the k-pairs kp = 4 KS (warp / 8) + 4 m + w4, m < KS; a warp
        // stores 8 rows x 4 words at a time (distinct banks in the K-major layout), and the phasors of
        // k and k + 1 advance by the exact 8-step phasor from one SFU start each.
        {
            const int w4 = tid & 3, tj = ((warp & 7) << 3) + ((tid >> 2) & 7), h = warp >> 3;
            const int tt = tj / CTC_PCH, j = tj % CTC_PCH;
            const bool valid = j < nc && blockIdx.x * CTC_TILES + tt < op.g.n_tiles;
            const int kp0 = h * KS * 4 + w4;
            float2 c0v = make_float2(0.f, 0.f), c1v = c0v, W8 = c0v;
            float sc = 1.0f;
            if (valid) {
                const PairTile& P = pt_s[buf + tj];
                c0v = tile_step_cis(P, 2 * kp0);
                c1v = tile_step_cis(P, 2 * kp0 + 1);
                W8 = p8_s[buf + tj];
                if (F16) sc = scale[j];
            }
            const float2* rr = rbuf + j * RB;
            // the word of k = 8 q + 2 w4 sits in K step q / 2, 8-column half q % 2
            const uint32_t row_re = kmaj_off(2 * tj, 2 * w4), row_im = kmaj_off(2 * tj + 1, 2 * w4);
            for (int m = 0; m < KS; ++m) {
                const int k = 2 * (kp0 + 4 * m);
                float2 v0 = make_float2(0.f, 0.f), v1 = v0;
                if (valid && k < K) {
                    const float4 rq = *reinterpret_cast<const float4*>(rr + k);   // r_k, r_{k+1}
                    float2 r0 = make_float2(rq.x, rq.y), r1 = make_float2(rq.z, rq.w);
                    if (op.pulse) {
                        r0 = cmul_conj(r0, op.pulse[k]);
                        if (k + 1 < K) r1 = cmul_conj(r1, op.pulse[k + 1]);
                    }
                    v0 = cmul(r0, c0v);
                    if (k + 1 < K) v1 = cmul(r1, c1v);
                    if (F16) {
                        v0.x *= sc;
                        v0.y *= sc;
                        v1.x *= sc;
                        v1.y *= sc;
                    }
                }
                if (valid) {
                    c0v = cmul(c0v, W8);
                    c1v = cmul(c1v, W8);
                }
                uint32_t hre, lre, him, lim;
                split2<F16>(v0.x, v1.x, hre, lre);
                split2<F16>(v0.y, v1.y, him, lim);
                const int q = h * KS + m;
                unsigned char* a0 = As + (q >> 1) * CTC_KSTEP_A + (q & 1) * 128;
                *reinterpret_cast<uint32_t*>(a0 + row_re) = hre;
                *reinterpret_cast<uint32_t*>(a0 + row_im) = him;
                *reinterpret_cast<uint32_t*>(a0 + KS * CTC_KSTEP_A + row_re) = lre;
                *reinterpret_cast<uint32_t*>(a0 + KS * CTC_KSTEP_A + row_im) = lim;
            }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0 && issue) {
            tc_fence_after();
            const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
            for (int s = 0; s < KS; ++s) {
                const uint64_t ahi = smem_desc(a_base + s * CTC_KSTEP_A);
                const uint64_t alo = smem_desc(a_base + (KS + s) * CTC_KSTEP_A);
                const uint64_t bhi = smem_desc(b_base + s * CTC_KSTEP_B);
                const uint64_t blo = smem_desc(b_base + (KS + s) * CTC_KSTEP_B);
                tc_mma(tbase, ahi, bhi, IDESC, s > 0 ? 1u : 0u);
                tc_mma(tbase, ahi, blo, IDESC, 1u);
                tc_mma(tbase, alo, bhi, IDESC, 1u);
            }
            tc_commit(bar);
        }
        if (c + 1 < n_chunks) load_r(c + 1);     // every thread is past its reads of rbuf
        if (c > 0) voxel_sum(c - 1);             // the tensor core works meanwhile
        __syncthreads();                         // craw and chunk c - 1's pair tiles are free
        if (c + 1 < n_chunks) load_tiles(c + 1);
        // the wait's outcome is made uniform over the CTA: on a timeout no thread reads TMEM, no further
        // MMA is issued and the iterate (or g) is left unwritten; the MMAs already committed get one more
        // bounded wait so that none is in flight when TMEM is released
        if (!__syncthreads_and(mbar_wait(bar, n_waits & 1u, op.wait_ns))) {
            if (issue) mbar_wait(bar, n_waits & 1u, op.wait_ns);
            ok = false;
            break;
        }
        ++n_waits;
        tc_fence_after();
        if (warp < 4) {                          // lanes 32 warp .. : rows (tile, pair, re/im)
            float d[32];
            tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16), d);
            const int row = tid;                 // tid < 128
            const int tt = row / (2 * CTC_PCH), j = (row / 2) % CTC_PCH, cc = row & 1;
            const float inv = F16 ? 1.0f / scale[j] : 1.0f;
            float* dst = reinterpret_cast<float*>(craw + (tt * CTC_PCH + j) * CRS) + cc;
#pragma unroll
            for (int l = 0; l < LT; ++l) dst[2 * l] = d[l] * inv;
        }
        cp_async_wait_all();                     // r of chunk c + 1
        tc_fence_before();
        __syncthreads();                         // craw, the pair tiles and r of the next chunk are ready
    }
    if (ok && n_chunks > 0) voxel_sum(n_chunks - 1);
    cp_async_wait_all();                         // no copy is left in flight (a timeout exits the loop early)
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

size_t adj_cheb_tc_smem_bytes(int K, int L)
{
    return (size_t)CtcSmem(K, L).total;
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
