// Tensor-core (tcgen05) form of the Chebyshev-expansion forward A_B s (the precision modes
// NFM_TC_BF16X3 / NFM_TC_FP16X3 for equally spaced frequencies).
//
// The expansion forward (op_cheb.cu) computes per (pair, tile) the moments
// m_l = sum_v u_v T_l(t_v) on the CUDA cores and then
//
//     S_k = sum_l (-j)^l b_l(k) m_l,      y_k += P_k S_k,   P_k = e^{-j 2 pi k df D_c / c}.
//
// b_l(k) is real and the same for every (pair, tile), so with m'_l = (-j)^l m_l
// (a re/im swap with signs) the first sum is one real GEMM D = A B^T per stage of
// 64 (pair, tile) items:
//
//     A[(g, c), l] = Re / Im m'_l(g)    M = 128 rows (64 items x re/im)
//     B[k, l]      = b_l(k)             N = the frequencies, padded to a multiple of 16
//     D[(g, c), k] = Re / Im S_k(g)     K = L padded to 16 (one or two K steps)
//
// Both operands are split x = hi + lo in BF16 (or FP16, each A row pair scaled by
// a power of two) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in FP32
// in tensor memory.  One thread issues the MMAs of stage q into one of two TMEM
// buffers and commits them to an mbarrier; while they run, every thread reads
// back stage q-1 (lane = row, a warp pair per lane quarter splits the
// columns), multiplies by the tile phasors P_k and adds into its rows of a
// shared accumulator, then computes the moments of stage q+1.  The moments,
// the phasors and the accumulation stay FP32 on the CUDA cores; only the
// 2 K L FMAs per (pair, tile) of the expansion move to the tensor core.
//
// CTA = 256 threads = 64 groups of 4 lanes; group g = (pair pl = g / TS, tile slot
// g % TS), PCH = 64 / TS pairs per CTA.  Chunk partials [chunk][slot][K] are summed
// by the deterministic chunk reduction as for the CUDA-core forward.
#include "nfm_kernels.cuh"
#include "cheb_device.cuh"
#include "tc_ptx.cuh"

namespace nfm {

namespace {

using namespace tc;

constexpr int FTC_THREADS = 256;
constexpr int FTC_G = 4;                           // lanes per (pair, tile) group
constexpr int FTC_NG = FTC_THREADS / FTC_G;        // 64 groups per stage
constexpr int FTC_M = 2 * FTC_NG;                  // 128 rows (group, re/im)
constexpr int FTC_KSTEP_A = FTC_M * 16 * 2;        // 4096 bytes: one K step (16 l) of A

__host__ __device__ constexpr int ftc_ksl(int LT) { return (LT + 15) / 16; }   // K steps over l
__host__ __device__ constexpr int ftc_n(int K) { return (K + 15) & ~15; }       // MMA N: frequencies, padded
__host__ __device__ constexpr int ftc_tmem_cols(int N)                           // two D buffers, power of 2
{
    return 2 * N <= 32 ? 32 : 2 * N <= 64 ? 64 : 2 * N <= 128 ? 128 : 256;
}

template <bool F16>
__device__ __forceinline__ uint32_t ftc_idesc(int N)
{
    // D FP32; A, B FP16 or BF16; both K-major; N >> 3 at bit 17, M >> 4 at bit 24
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(FTC_M >> 4) << 24);
}

// per (pair, tile) item of a stage, handed from the moment phase to the read-back of that stage
struct __align__(16) FtcSlot {
    float S_hi, S_lo;      // frac(df D_c / c) as hi + lo (the tile phasor P_k = e^{-j 2 pi k (S_hi + S_lo)})
    float w_re, w_im;      // e^{+j 2 pi (S_hi + S_lo)}: one step of the conjugate phasor
    float inv_scale;       // 1 / (power-of-two scale of the item's A rows)
    float pad0, pad1, pad2;
};

struct FtcSmem {   // byte offsets of the dynamic shared-memory regions
    int b, a, acc, voff, s, ant, pair, slot, bar, tslot, total;
    __host__ __device__ FtcSmem(int LT, int K, int TS)
    {
        const int KSL = ftc_ksl(LT), N = ftc_n(K);
        b = 0;                                                   // [split 2][KSL][N rows x 32 B]
        a = (b + 2 * KSL * N * 32 + 1023) & ~1023;               // [buf 2][split 2][KSL][4096]
        acc = a + 2 * 2 * KSL * FTC_KSTEP_A;                     // [64 groups][N + 1] float2 (odd stride)
        voff = (acc + FTC_NG * (N + 1) * 8 + 15) & ~15;          // [128] VoxelOffset
        s = voff + TILE_V * 16;                                  // [buf 2][TS][128] float2
        ant = s + 2 * TS * TILE_V * 8;                           // [buf 2][64][2] AntTile
        pair = ant + 2 * FTC_NG * 2 * (int)sizeof(AntTile);      // [64] int
        slot = pair + FTC_NG * 4;                                // [buf 2][64] FtcSlot
        bar = slot + 2 * FTC_NG * (int)sizeof(FtcSlot);          // two mbarriers
        tslot = bar + 16;
        total = tslot + 16;
    }
};

// (cos, sin)(2 pi k (S_hi + S_lo)) with k S_hi split exactly (one rounding at |x| <= 1/2), SFU sine/cosine
__device__ __forceinline__ float2 slot_cis(float S_hi, float S_lo, int k)
{
    const float kf = (float)k;
    const float p = __fmul_rn(kf, S_hi);        // rounded product: its error e is added back below
    const float e = fmaf(kf, S_hi, -p);
    const float ph = (p - rintf(p)) + fmaf(kf, S_lo, e);
    return cis_turns_sfu(ph);
}

}  // namespace

template <int LT, bool F16>
__global__ void __launch_bounds__(FTC_THREADS, 2) fwd_cheb_tc_kernel(OpDesc op, ChebDesc cd, FwdArgs a)
{
    constexpr int LS = (LT + 3) & ~3;        // row stride of the coefficient table in global memory
    constexpr int KSL = ftc_ksl(LT);
    extern __shared__ __align__(1024) unsigned char smem[];
    const int K = op.K;
    const int N = ftc_n(K);
    const int AS = N + 1;                    // accumulator row stride (float2)
    const int PCH = a.VS;                    // pairs per CTA: 16, 32 or 64
    const int TS = FTC_NG / PCH;             // tiles per stage
    const FtcSmem L(LT, K, TS);
    unsigned char* Bs = smem + L.b;
    unsigned char* As = smem + L.a;
    float2* acc = reinterpret_cast<float2*>(smem + L.acc);
    VoxelOffset* voff = reinterpret_cast<VoxelOffset*>(smem + L.voff);
    float2* s_st = reinterpret_cast<float2*>(smem + L.s);
    AntTile* ant_st = reinterpret_cast<AntTile*>(smem + L.ant);
    int* pair_s = reinterpret_cast<int*>(smem + L.pair);
    FtcSlot* slots = reinterpret_cast<FtcSlot*>(smem + L.slot);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);

    const int tid = threadIdx.x;
    const int warp = tid / 32, lane = tid % 32;
    const int g = tid / FTC_G, ln = tid % FTC_G;
    const int pl = g / TS, sl = g % TS;
    const unsigned gmask = 0xFu << (lane & ~3);
    const int pair_base = blockIdx.x * PCH;
    const int chunk = blockIdx.y;
    const int t_begin = chunk * a.tiles_base + min(chunk, a.tiles_rem);
    const int t_end = t_begin + a.tiles_base + (chunk < a.tiles_rem ? 1 : 0);
    const int n_stages = (t_end - t_begin + TS - 1) / TS;
    const uint32_t idesc = ftc_idesc<F16>(N);
    const bool issue = !(op.hooks & HOOK_TC_SKIP_ISSUE);

    if (warp == 0) {
        tmem_alloc(tslot, (uint32_t)ftc_tmem_cols(N));
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    // B = b_l(k): rows k < N (zero beyond K), l pairs per 32-bit word, zero for l >= LT (constant table:
    // read before the wait on the previous kernel)
    for (int e = tid; e < N * 8 * KSL; e += FTC_THREADS) {
        const int k = e / (8 * KSL), l = 2 * (e % (8 * KSL));
        const float b0 = (k < K && l < LT) ? cd.coef[k * LS + l] : 0.f;
        const float b1 = (k < K && l + 1 < LT) ? cd.coef[k * LS + l + 1] : 0.f;
        uint32_t hi, lo;
        split2<F16>(b0, b1, hi, lo);
        const int s = l / 16, kk = l % 16;
        *reinterpret_cast<uint32_t*>(Bs + (0 * KSL + s) * N * 32 + kmaj_off(k, kk)) = hi;
        *reinterpret_cast<uint32_t*>(Bs + (1 * KSL + s) * N * 32 + kmaj_off(k, kk)) = lo;
    }
    for (int v = tid; v < TILE_V; v += FTC_THREADS)
        voff[v] = voxel_offset(op.g, v % TILE_X, (v / TILE_X) % TILE_Y, v / (TILE_X * TILE_Y));
    for (int i = tid; i < FTC_NG * AS; i += FTC_THREADS)   // the accumulator rows start at zero
        acc[i] = make_float2(0.f, 0.f);
    if (tid < PCH) {
        const int sp = pair_base + tid;
        int pair = sp < a.n_pairs ? a.pairs[sp] : -1;
        if (sp < a.n_pairs && (pair < 0 || pair >= op.P)) {   // flagged; pair 0 keeps every access in bounds
            atomicOr(op.err, ERRF_PAIR);
            pair = 0;
        }
        pair_s[tid] = pair;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    auto load_geom = [&](int q) {            // the two antenna-tile rows of every group
        const int buf = q & 1;
        for (int i = tid; i < FTC_NG * 6; i += FTC_THREADS) {
            const int gi = i / 6, part = i % 6;
            const int tile = t_begin + q * TS + gi % TS;
            const int pair = pair_s[gi / TS];
            if (tile < t_end && pair >= 0) {
                const AntTile *at, *ar;
                pair_rows(op, pair, tile, at, ar);
                AntTile* dst = ant_st + (buf * FTC_NG + gi) * 2 + (part < 3 ? 0 : 1);
                cp_async_16(reinterpret_cast<float4*>(dst) + part % 3,
                            reinterpret_cast<const float4*>(part < 3 ? at : ar) + part % 3);
            }
        }
    };
    auto load_s = [&](int q) {               // the stage's scene values (zero outside the grid)
        const int buf = q & 1;
        for (int e = tid; e < TS * TILE_V; e += FTC_THREADS) {
            const int st = e / TILE_V, v = e % TILE_V;
            const int tile = t_begin + q * TS + st;
            if (tile >= t_end) continue;
            int tx, ty, tz;
            tile_coords(op.g, tile, tx, ty, tz);
            const int ix = tx * TILE_X + v % TILE_X, iy = ty * TILE_Y + (v / TILE_X) % TILE_Y,
                      iz = tz * TILE_Z + v / (TILE_X * TILE_Y);
            const bool in = ix < op.g.nx && iy < op.g.ny && iz < op.g.nz;
            const float2* src = in ? a.s + ((size_t)iz * op.g.ny + iy) * op.g.nx + ix : a.s;
            cp_async_8(s_st + (buf * TS + st) * TILE_V + v, src, in);
        }
    };

    // moments of stage q into A[q & 1] (rows 2g, 2g + 1) and the item's slot record
    auto moments = [&](int q) {
        const int buf = q & 1;
        const int tile = t_begin + q * TS + sl;
        const bool valid = tile < t_end && pair_s[pl] >= 0;     // uniform over the group's lanes
        float mr[LT], mi[LT];
#pragma unroll
        for (int l = 0; l < LT; ++l) mr[l] = mi[l] = 0.f;
        PairTile P;
        if (valid) {
            const AntTile* ap = ant_st + (buf * FTC_NG + g) * 2;
            P = fold_pair_tile(ap[0], ap[1]);
            const float2* sb = s_st + (buf * TS + sl) * TILE_V;
#pragma unroll 2
            for (int i = 0; i < TILE_V / FTC_G; ++i) {
                const int v = ln + FTC_G * i;
                const float2 sv = sb[v];
                const ChebVoxel cv = cheb_voxel(P, voff[v], cd.fc_hi, cd.fc_lo);
                const float2 c0 = cis_turns_sfu(cv.th0);
                const float2 u = cmul_conj(make_float2(cv.amp * sv.x, cv.amp * sv.y), c0);
                const float t = cv.delta * cd.tau;
                const float t2 = t + t;
                mr[0] += u.x;
                mi[0] += u.y;
                mr[1] = fmaf(u.x, t, mr[1]);
                mi[1] = fmaf(u.y, t, mi[1]);
                float Tp = 1.f, Tc = t;
#pragma unroll
                for (int l = 2; l < LT; ++l) {
                    const float Tn = fmaf(t2, Tc, -Tp);
                    mr[l] = fmaf(u.x, Tn, mr[l]);
                    mi[l] = fmaf(u.y, Tn, mi[l]);
                    Tp = Tc;
                    Tc = Tn;
                }
            }
#pragma unroll
            for (int w = 1; w < FTC_G; w *= 2) {
#pragma unroll
                for (int l = 0; l < LT; ++l) {
                    mr[l] += __shfl_xor_sync(gmask, mr[l], w);
                    mi[l] += __shfl_xor_sync(gmask, mi[l], w);
                }
            }
        }
        float sc = 1.f, inv = 1.f;
        if (F16) {                           // rows scaled so that every value is below 1 in magnitude
            float mx = 0.f;
#pragma unroll
            for (int l = 0; l < LT; ++l) mx = fmaxf(mx, fmaxf(fabsf(mr[l]), fabsf(mi[l])));
            if (mx > 0.f) {
                int ex;
                frexpf(mx, &ex);
                sc = ldexpf(1.0f, -ex);
                inv = ldexpf(1.0f, ex);
            }
        }
        // m'_l = (-j)^l m_l: l % 4 = 0: (mr, mi), 1: (mi, -mr), 2: (-mr, -mi), 3: (-mi, mr); quads of l go
        // round robin to the group's lanes (compile-time register indices, predicated stores)
        unsigned char* Ab = As + buf * (2 * KSL * FTC_KSTEP_A);
        const int row = 2 * g;
#pragma unroll
        for (int l = 0; l < 16 * KSL; l += 2) {
            if (((l >> 2) & 3) != ln) continue;
            float re[2], im[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ll = l + h;
                const float xr = ll < LT ? mr[ll < LT ? ll : 0] : 0.f;
                const float xi = ll < LT ? mi[ll < LT ? ll : 0] : 0.f;
                const int r4 = ll & 3;
                re[h] = (r4 == 0 ? xr : r4 == 1 ? xi : r4 == 2 ? -xr : -xi) * sc;
                im[h] = (r4 == 0 ? xi : r4 == 1 ? -xr : r4 == 2 ? -xi : xr) * sc;
            }
            uint32_t hre, lre, him, lim;
            split2<F16>(re[0], re[1], hre, lre);
            split2<F16>(im[0], im[1], him, lim);
            unsigned char* a0 = Ab + (l >> 4) * FTC_KSTEP_A;
            const int kk = l & 15;
            *reinterpret_cast<uint32_t*>(a0 + kmaj_off(row, kk)) = hre;
            *reinterpret_cast<uint32_t*>(a0 + kmaj_off(row + 1, kk)) = him;
            *reinterpret_cast<uint32_t*>(a0 + KSL * FTC_KSTEP_A + kmaj_off(row, kk)) = lre;
            *reinterpret_cast<uint32_t*>(a0 + KSL * FTC_KSTEP_A + kmaj_off(row + 1, kk)) = lim;
        }
        if (ln == 0) {
            FtcSlot so;
            so.S_hi = valid ? P.S_hi : 0.f;
            so.S_lo = valid ? P.S_lo : 0.f;
            float2 w = make_float2(1.f, 0.f);
            if (valid) {                     // Taylor-series phasor (error ~1e-7): it is repeated below
                const PairTile& Pr = P;
                w = tile_step_cis_exact(Pr, 1);
            }
            so.w_re = w.x;
            so.w_im = w.y;
            so.inv_scale = inv;
            so.pad0 = so.pad1 = so.pad2 = 0.f;
            slots[buf * FTC_NG + g] = so;
        }
    };

    auto issue_mma = [&](int q) {            // one thread: D[q & 1] = A[q & 1] B^T in three split products
        const int buf = q & 1;
        tc_fence_after();
        const uint32_t d = tbase + (uint32_t)(buf * N);
        const uint32_t a_base = smem_u32(As + buf * (2 * KSL * FTC_KSTEP_A)), b_base = smem_u32(Bs);
#pragma unroll
        for (int s = 0; s < KSL; ++s) {
            const uint64_t ahi = smem_desc(a_base + s * FTC_KSTEP_A);
            const uint64_t alo = smem_desc(a_base + (KSL + s) * FTC_KSTEP_A);
            const uint64_t bhi = smem_desc(b_base + s * N * 32);
            const uint64_t blo = smem_desc(b_base + (KSL + s) * N * 32);
            tc_mma(d, ahi, bhi, idesc, s > 0 ? 1u : 0u);
            tc_mma(d, ahi, blo, idesc, 1u);
            tc_mma(d, alo, bhi, idesc, 1u);
        }
        tc_commit(&bar[buf]);
    };

    // stage qe: wait for its MMAs, read D back (lane = row; warps w and w + 4 take the two column halves of
    // one lane quarter), exchange re/im with the neighbouring lane (rows 2g, 2g + 1), multiply by the tile
    // phasor P_k and add into the item's accumulator row; false on a timed-out wait (uniform over the CTA)
    auto readback = [&](int qe) -> bool {
        const int buf = qe & 1;
        if (!__syncthreads_and(mbar_wait(&bar[buf], (uint32_t)((qe >> 1) & 1), op.wait_ns))) return false;
        tc_fence_after();
        const int quarter = warp & 3, half = warp >> 2;
        const int row = 32 * quarter + lane, gg = row >> 1, c = row & 1;
        const FtcSlot so = slots[buf * FTC_NG + gg];
        const float2 w = make_float2(so.w_re, so.w_im);
        const int NH = N / 2;
        float2* accg = acc + gg * AS;
        const uint32_t taddr = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * N + half * NH);
        for (int cb = 0; cb < NH; cb += 8) {
            float d[8];
            tmem_ld8(taddr + (uint32_t)cb, d);
            // c = 0 keeps columns cb .. cb + 3 (its re, the neighbour's im); c = 1 keeps cb + 4 .. cb + 7
            float o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = __shfl_xor_sync(0xffffffffu, c ? d[i] : d[4 + i], 1);
            const int k0 = half * NH + cb + 4 * c;
            float2 ph = slot_cis(so.S_hi, so.S_lo, k0);   // scaled by the item's 1/scale (w has unit modulus)
            ph.x *= so.inv_scale;
            ph.y *= so.inv_scale;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float sr = c ? o[i] : d[i];
                const float si = c ? d[4 + i] : o[i];
                const int k = k0 + i;
                if (k < K) {                 // y_k += P_k S_k, P_k = (ph.x, -ph.y); the rows start at zero
                    float2 y = accg[k];
                    y.x = fmaf(ph.x, sr, fmaf(ph.y, si, y.x));
                    y.y = fmaf(ph.x, si, fmaf(-ph.y, sr, y.y));
                    accg[k] = y;
                }
                ph = cmul(ph, w);
            }
        }
        return true;
    };

    if (n_stages > 0) load_geom(0);
    pdl_wait();                              // s may come from the previous kernel
    if (n_stages > 0) {
        load_s(0);
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();
    bool ok = true;
    int committed = 0, failed = 0;           // stages whose MMAs were committed; the stage whose wait ran out
    for (int q = 0; q < n_stages; ++q) {
        if (q + 1 < n_stages) {
            load_geom(q + 1);
            load_s(q + 1);
            cp_async_commit();
        }
        moments(q);
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (issue) {
            if (tid == 0) issue_mma(q);
            committed = q + 1;
        }
        if (q > 0 && !readback(q - 1)) {
            ok = false;
            failed = q - 1;
            break;
        }
        cp_async_wait_all();
        tc_fence_before();
        __syncthreads();
    }
    if (ok && n_stages > 0 && !readback(n_stages - 1)) {
        ok = false;
        failed = n_stages - 1;
    }
    cp_async_wait_all();
    if (!ok) {                               // let every committed MMA finish (bounded) before TMEM goes
        for (int qq = failed; qq < committed; ++qq) mbar_wait(&bar[qq & 1], (uint32_t)((qq >> 1) & 1), op.wait_ns);
        if (tid == 0) atomicOr(op.err, ERRF_TIMEOUT);
    }
    pdl_launch_dependents();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, (uint32_t)ftc_tmem_cols(N));
    }
    if (!ok) return;
    // sum the TS slots of each pair in slot order (the rows start at zero) and write the chunk partial
    for (int e = tid; e < PCH * K; e += FTC_THREADS) {
        const int p = e / K, k = e - (e / K) * K;
        const int sp = pair_base + p;
        if (sp >= a.n_pairs) continue;
        const float2* col = acc + (p * TS) * AS + k;
        float2 sum = col[0];
        for (int t = 1; t < TS; ++t) {
            const float2 x = col[t * AS];
            sum.x += x.x;
            sum.y += x.y;
        }
        a.partial[((size_t)chunk * a.n_slots + sp) * K + k] = sum;
    }
}

size_t fwd_cheb_tc_smem_bytes(int LT, int K, int pch)
{
    return (size_t)FtcSmem(LT, K, FTC_NG / pch).total;
}

template <bool F16>
static const void* fwd_cheb_tc_ptr_f(int LT)
{
    switch (LT) {
    case 10: return (const void*)fwd_cheb_tc_kernel<10, F16>;
    case 12: return (const void*)fwd_cheb_tc_kernel<12, F16>;
    case 14: return (const void*)fwd_cheb_tc_kernel<14, F16>;
    case 16: return (const void*)fwd_cheb_tc_kernel<16, F16>;
    case 18: return (const void*)fwd_cheb_tc_kernel<18, F16>;
    case 20: return (const void*)fwd_cheb_tc_kernel<20, F16>;
    case 22: return (const void*)fwd_cheb_tc_kernel<22, F16>;
    case 24: return (const void*)fwd_cheb_tc_kernel<24, F16>;
    case 26: return (const void*)fwd_cheb_tc_kernel<26, F16>;
    case 28: return (const void*)fwd_cheb_tc_kernel<28, F16>;
    case 30: return (const void*)fwd_cheb_tc_kernel<30, F16>;
    case 32: return (const void*)fwd_cheb_tc_kernel<32, F16>;
    default: return nullptr;
    }
}

const void* fwd_cheb_tc_kernel_ptr(int LT, bool f16)
{
    return f16 ? fwd_cheb_tc_ptr_f<true>(LT) : fwd_cheb_tc_ptr_f<false>(LT);
}

cudaError_t launch_fwd_cheb_tc(const OpDesc& op, const ChebDesc& cd, const FwdArgs& a, dim3 grid, bool f16,
                               size_t smem, cudaStream_t st)
{
    const void* fn = fwd_cheb_tc_kernel_ptr(cd.L, f16);
    if (!fn || op.K > GEN_MAX_K || (a.VS != 16 && a.VS != 32 && a.VS != 64)) return cudaErrorInvalidValue;
    void* args[] = {(void*)&op, (void*)&cd, (void*)&a};
    return launch_pdl(fn, grid, dim3(FTC_THREADS), smem, st, args);
}

}  // namespace nfm
