// Minibatch forward operator y = A_B s on CUDA cores (Eq. 2 rows of a pair list).
//
// Work split: blockIdx.x = group of FWD_PC pairs, blockIdx.y = chunk of voxel
// tiles (a contiguous tile range).  Each CTA writes a partial spectrum
// [FWD_PC][K] for its chunk; fwd_reduce_kernel sums the chunks in a fixed
// order, so the result does not depend on scheduling.
//
// The CTA walks its tiles in stages of half a tile (64 voxels).  For a stage
// it loads s and the FWD_PC (pair, tile) constants, then builds for every
// (voxel, pair) the block start values
//        U[k1] = amp s exp(-j 2 pi (f0 + k1 K2 df) D / c)      (k1 < K1)
// and the fine step w = exp(-j 2 pi df D / c) in shared memory.  Warp p
// (one pair) then walks the stage's voxels, lane (k1, vs) two voxels at a
// time, and accumulates the K2 frequencies of block k1.  The terms u w^k come
// from the real-coefficient recurrence t_{k+1} = 2 cos(theta) t_k - t_{k-1}
// (4 FP32 lane-instructions per (row, voxel) element with the accumulation).
// That recurrence amplifies rounding by 1/|sin theta|, so for (pair, tile)
// whose step phase lies within 1/8 turn of 0 or 1/2 the sequence is generated
// with w' = -j w (a quarter turn more per step) and the factor j^k is undone
// exactly by permuting real and imaginary parts in the accumulation.  Stages
// are software pipelined with one barrier each: iteration q loads stage q+2,
// builds stage q+1 and consumes stage q, so every warp shares both kinds of work.
#include "nfm_kernels.cuh"

namespace nfm {

constexpr int FWD_SV = TILE_V / 2;   // voxels per stage: half a tile (8 x 4 x 2)

// Shared-memory layout of one stage buffer: U [SV][VSTR] with U[v][pair][k1]
// at v*VSTR + pair*K1 + k1, then W [SV][PC+1].  VSTR = 9 K1 puts the K1-wide
// groups a warp reads for consecutive voxels on distinct banks.
template <int K1>
struct FwdSmem {
    static constexpr int VSTR = 9 * K1;
    static constexpr int WSTR = FWD_PC + 1;
    static constexpr int BUF = FWD_SV * VSTR + FWD_SV * WSTR;
};

// acc[k] += i^k t (rotated frame) or acc[k] += t, for k = j mod 4.
template <bool ROT, int J>
__device__ __forceinline__ void acc_add(float2& acc, float tx, float ty)
{
    if (!ROT || (J & 3) == 0) { acc.x += tx; acc.y += ty; }
    else if ((J & 3) == 1) { acc.x -= ty; acc.y += tx; }
    else if ((J & 3) == 2) { acc.x -= tx; acc.y -= ty; }
    else { acc.x += ty; acc.y -= tx; }
}

// K2 terms of u w'^k for two voxels a, b by the real three-term recurrence
// t_{k+1} = 2 cos(theta') t_k - t_{k-1} (w' = exp(-j theta'), |w'| = 1).
template <bool ROT>
__device__ __forceinline__ void run_block(float2 (&acc)[K2], float2 ta0, float2 wa, float2 tb0, float2 wb)
{
    const float ca = 2.0f * wa.x, cb = 2.0f * wb.x;
    float2 ta1 = cmul(ta0, wa), tb1 = cmul(tb0, wb);
    acc_add<ROT, 0>(acc[0], ta0.x + tb0.x, ta0.y + tb0.y);
    acc_add<ROT, 1>(acc[1], ta1.x + tb1.x, ta1.y + tb1.y);
#pragma unroll
    for (int j = 2; j < K2; ++j) {
        const float2 ta2 = make_float2(fmaf(ca, ta1.x, -ta0.x), fmaf(ca, ta1.y, -ta0.y));
        const float2 tb2 = make_float2(fmaf(cb, tb1.x, -tb0.x), fmaf(cb, tb1.y, -tb0.y));
        const float sx = ta2.x + tb2.x, sy = ta2.y + tb2.y;
        switch (j & 3) {
        case 0: acc_add<ROT, 0>(acc[j], sx, sy); break;
        case 1: acc_add<ROT, 1>(acc[j], sx, sy); break;
        case 2: acc_add<ROT, 2>(acc[j], sx, sy); break;
        default: acc_add<ROT, 3>(acc[j], sx, sy); break;
        }
        ta0 = ta1; ta1 = ta2;
        tb0 = tb1; tb1 = tb2;
    }
}

template <int K1>
__global__ void __launch_bounds__(256, 3) fwd_partial_kernel(OpDesc op, FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int PC = FWD_PC;
    constexpr int SV = FWD_SV;
    constexpr int VSTR = FwdSmem<K1>::VSTR;
    constexpr int WSTR = FwdSmem<K1>::WSTR;
    constexpr int BUF = FwdSmem<K1>::BUF;
    constexpr int VS = 32 / K1;             // voxel subsets per warp (lanes beyond VS*K1 idle)
    const int nt = blockDim.x;              // 256: one warp per pair of the group
    const int tid = threadIdx.x;
    const int group = blockIdx.x;
    const int chunk = blockIdx.y;

    float2* ubuf = reinterpret_cast<float2*>(smem);                     // [2][BUF]
    VoxelOffset* voff = reinterpret_cast<VoxelOffset*>(ubuf + 2 * BUF);  // [TILE_V]
    AntTile* ant_st = reinterpret_cast<AntTile*>(voff + TILE_V);        // [3][PC][2] (TX, RX)
    float2* s_st = reinterpret_cast<float2*>(ant_st + 3 * PC * 2);      // [3][SV]
    int* pair_s = reinterpret_cast<int*>(s_st + 3 * SV);                // [PC]
    int* rot_s = pair_s + PC;                                           // [2][PC]

    // consume role: warp = pair, lane = (k1, voxel subset)
    const int p = tid / 32;
    const int lane = tid % 32;
    const int k1 = lane % K1;
    const int vs = lane / K1;

    float2 acc[K2];
#pragma unroll
    for (int i = 0; i < K2; ++i) acc[i] = make_float2(0.f, 0.f);

    const int t_begin = chunk * a.tiles_base + min(chunk, a.tiles_rem);
    const int t_end = t_begin + a.tiles_base + (chunk < a.tiles_rem ? 1 : 0);
    const int q0 = 2 * t_begin;             // stage = (tile, half)
    const int nq = 2 * (t_end - t_begin);

    for (int v = tid; v < TILE_V; v += nt)
        voff[v] = voxel_offset(op.g, v % TILE_X, (v / TILE_X) % TILE_Y, v / (TILE_X * TILE_Y));
    pdl_wait();                              // s and pairs may come from the previous kernel
    if (tid < PC) {
        int slot = group * PC + tid;
        pair_s[tid] = slot < a.n_pairs ? a.pairs[slot] : -1;
    }
    __syncthreads();

    // asynchronous loads of a stage: its s values and the two AntTile rows per pair
    auto load_small = [&](int q) {
        const int sidx = q0 + q;
        const int tile = sidx >> 1, half = sidx & 1;
        int tx, ty, tz;
        tile_coords(op.g, tile, tx, ty, tz);
        float2* sb = s_st + (q % 3) * SV;
        for (int v = tid; v < SV; v += nt) {
            int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y) + 2 * half;
            int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
            bool in = ix < op.g.nx && iy < op.g.ny && iz < op.g.nz;
            const float2* src = in ? a.s + ((size_t)iz * op.g.ny + iy) * op.g.nx + ix : a.s;
            cp_async_8(sb + v, src, in);
        }
        if (tid < PC * 6) {                   // 2 rows x 48 B = 6 chunks of 16 B per pair
            const int i = tid / 6, part = tid % 6;
            const int pair = pair_s[i];
            const AntTile *at, *ar;
            pair_rows(op, pair < 0 ? 0 : pair, tile, at, ar);
            const AntTile* src = part < 3 ? at : ar;
            AntTile* dst = ant_st + ((q % 3) * PC + i) * 2 + (part < 3 ? 0 : 1);
            cp_async_16(reinterpret_cast<float4*>(dst) + part % 3, reinterpret_cast<const float4*>(src) + part % 3);
        }
        cp_async_commit();
    };

    // block start values U[k1] and the step w' of every (voxel, pair) of a stage;
    // w' is w turned by a quarter turn per step when the pair's step phase is
    // near 0 or 1/2 turn, so the recurrence never divides by a small sine
    auto stage = [&](int q) {
        const int half = (q0 + q) & 1;
        float2* U = ubuf + (q & 1) * BUF;
        float2* Wf = U + SV * VSTR;
        const float2* sb = s_st + (q % 3) * SV;
        const int i = tid % PC;                      // every item of this thread has pair i
        const bool live = pair_s[i] >= 0;
        const AntTile* aq = ant_st + ((q % 3) * PC + i) * 2;
        const PairTile P = fold_pair_tile(aq[0], aq[1]);
        const float sa = fabsf(P.S_hi);
        const bool rot = sa < 0.125f || sa > 0.375f;
        if (tid < PC) rot_s[(q & 1) * PC + i] = rot;
#pragma unroll 2
        for (int item = tid; item < SV * PC; item += nt) {
            const int v = item / PC;
            float2* Up = U + v * VSTR + i * K1;
            if (!live) {
#pragma unroll
                for (int j = 0; j < K1; ++j) Up[j] = make_float2(0.f, 0.f);
                Wf[v * WSTR + i] = make_float2(1.f, 0.f);
                continue;
            }
            const float2 sv = sb[v];
            const VoxelOffset o = voff[v + SV * half];
            const PVGeom gv = pair_voxel(P, o, op.ph);
            const float2 c0 = cis_turns_sfu(gv.th0);
            const float2 cw = cis_turns(gv.dth);
            float2 u = cmul_conj(make_float2(gv.amp * sv.x, gv.amp * sv.y), c0);
            Up[0] = u;
            if (K1 > 1) {
                const float2 cW = cis_turns_sfu(gv.dth2);
                const float2 Wc = make_float2(cW.x, -cW.y);
#pragma unroll
                for (int j = 1; j < K1; ++j) {
                    u = cmul(u, Wc);
                    Up[j] = u;
                }
            }
            // w = (c, -s); turned: -j w = (-s, -c)
            Wf[v * WSTR + i] = rot ? make_float2(-cw.y, -cw.x) : make_float2(cw.x, -cw.y);
        }
    };

    // three-term recurrence over the K2 frequencies of block k1, two voxels at a time
    auto consume = [&](int q) {
        if (vs >= VS) return;
        const float2* U = ubuf + (q & 1) * BUF;
        const float2* Wf = U + SV * VSTR;
        const bool rot = rot_s[(q & 1) * PC + p] != 0;   // warp-uniform
        int v = vs;
        for (; v + VS < SV; v += 2 * VS) {
            const float2 ta = U[v * VSTR + p * K1 + k1];
            const float2 wa = Wf[v * WSTR + p];
            const float2 tb = U[(v + VS) * VSTR + p * K1 + k1];
            const float2 wb = Wf[(v + VS) * WSTR + p];
            if (rot) run_block<true>(acc, ta, wa, tb, wb);
            else run_block<false>(acc, ta, wa, tb, wb);
        }
        if (v < SV) {
            const float2 ta = U[v * VSTR + p * K1 + k1];
            const float2 wa = Wf[v * WSTR + p];
            const float2 zero = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f);
            if (rot) run_block<true>(acc, ta, wa, zero, one);
            else run_block<false>(acc, ta, wa, zero, one);
        }
    };

    // pipeline: iteration q loads stage q+2, builds stage q+1, consumes stage q
    if (nq > 0) {
        load_small(0);
        if (nq > 1) load_small(1);
        cp_async_wait_all();
        __syncthreads();
        stage(0);
        __syncthreads();
        for (int q = 0; q < nq; ++q) {
            if (q + 2 < nq) load_small(q + 2);
            if (q + 1 < nq) stage(q + 1);
            consume(q);
            cp_async_wait_all();
            __syncthreads();
        }
    }
    pdl_launch_dependents();

    // reduce the VS voxel subsets in a fixed order, then write the partial
    float2* red = reinterpret_cast<float2*>(smem);        // [PC][VS][K1*K2]
    constexpr int KB = K1 * K2;
    if (vs < VS) {
#pragma unroll
        for (int j = 0; j < K2; ++j) red[((p * VS + vs) * K1 + k1) * K2 + j] = acc[j];
    }
    __syncthreads();
    for (int o = tid; o < PC * KB; o += nt) {
        int i = o / KB;
        int kk = o - i * KB;
        int slot = group * PC + i;
        if (kk >= op.K || slot >= a.n_pairs) continue;
        float2 sum = red[(i * VS) * KB + kk];
        for (int u = 1; u < VS; ++u) {
            float2 x = red[(i * VS + u) * KB + kk];
            sum.x += x.x;
            sum.y += x.y;
        }
        a.partial[((size_t)chunk * a.n_slots + slot) * op.K + kk] = sum;
    }
}

size_t fwd_smem_bytes(int K1, int nt)
{
    const size_t buf = (size_t)FWD_SV * 9 * K1 + FWD_SV * (FWD_PC + 1);
    size_t stage = 2 * buf * sizeof(float2) + TILE_V * sizeof(VoxelOffset) + 3 * FWD_PC * 2 * sizeof(AntTile) +
                   3 * FWD_SV * sizeof(float2) + 3 * FWD_PC * sizeof(int);
    size_t red = (size_t)nt * K2 * sizeof(float2);
    return stage > red ? stage : red;
}

const void* fwd_kernel_ptr(int K1)
{
    switch (K1) {
    case 1: return (const void*)fwd_partial_kernel<1>;
    case 2: return (const void*)fwd_partial_kernel<2>;
    case 3: return (const void*)fwd_partial_kernel<3>;
    case 4: return (const void*)fwd_partial_kernel<4>;
    case 5: return (const void*)fwd_partial_kernel<5>;
    case 6: return (const void*)fwd_partial_kernel<6>;
    case 7: return (const void*)fwd_partial_kernel<7>;
    case 8: return (const void*)fwd_partial_kernel<8>;
    default: return nullptr;
    }
}

cudaError_t launch_fwd_partial(const OpDesc& op, const FwdArgs& a, dim3 grid, int nt, size_t smem,
                               cudaStream_t st)
{
    const void* fn = fwd_kernel_ptr(op.K1);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&op, (void*)&a};
    return launch_pdl(fn, grid, dim3(nt), smem, st, args);
}

// Sum the chunk partials in chunk order (fixed), apply p(f_k), and optionally
// subtract the observed rows: out[slot*K + k] = p_k sum_c partial[c][slot][k] - y[pair*K + k].
// CTA = RED_OUT outputs x 32 chunk lanes; lane y sums chunks y, y+32, ... in that
// order, then the 32 lane sums are added in lane order.
constexpr int RED_OUT = 4;
__device__ __forceinline__ void fwd_reduce_body(const OpDesc& op, const ReduceArgs& a, int block)
{
    constexpr int UN = 8;                 // loads in flight per thread
    __shared__ float2 red[32][RED_OUT + 1];
    const int ox = threadIdx.x % RED_OUT, cy = threadIdx.x / RED_OUT;
    const int o = block * RED_OUT + ox;
    const size_t stride = (size_t)a.n_slots * op.K;
    pdl_wait();
    float2 s = make_float2(0.f, 0.f);
    if (o < a.n_out) {
        for (int c0 = cy; c0 < a.n_chunks; c0 += 32 * UN) {
            float2 x[UN];
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int c = c0 + 32 * u;
                x[u] = c < a.n_chunks ? a.partial[NFM_IDX((size_t)c * stride + o, a.partial_elems, op.err)]
                                      : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                s.x += x[u].x;
                s.y += x[u].y;
            }
        }
    }
    red[cy][ox] = s;
    __syncthreads();
    if (cy == 0 && o < a.n_out) {
        float2 t = red[0][ox];
#pragma unroll
        for (int y = 1; y < 32; ++y) {
            t.x += red[y][ox].x;
            t.y += red[y][ox].y;
        }
        const int k = o % op.K;
        if (op.pulse) t = cmul(op.pulse[k], t);
        if (a.y_obs) {
            int pair = a.pairs[o / op.K];
            if (pair < 0 || pair >= op.P) {
                atomicOr(op.err, ERRF_PAIR);
                pair = 0;
            }
            const float2 yo = a.y_obs[NFM_IDX((size_t)pair * op.K + k, op.m_rows, op.err)];
            t.x -= yo.x;
            t.y -= yo.y;
            if (a.fmask && !a.fmask[k]) t = make_float2(0.f, 0.f);
        }
        a.out[o] = t;
    }
    pdl_launch_dependents();
}

__global__ void __launch_bounds__(RED_OUT * 32) fwd_reduce_kernel(OpDesc op, ReduceArgs a)
{
    fwd_reduce_body(op, a, blockIdx.x);
}

// One launch over the chunk reductions of several scenes: CTA b belongs to the item with the largest
// cta0 <= b (items sorted by cta0, the first at 0).
__global__ void __launch_bounds__(RED_OUT * 32) fwd_reduce_multi_kernel(const MultiRedItem* __restrict__ items,
                                                                        int n_items)
{
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].cta0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const OpDesc op = items[lo].op;
    const ReduceArgs a = items[lo].a;
    fwd_reduce_body(op, a, (int)blockIdx.x - items[lo].cta0);
}

cudaError_t launch_fwd_reduce_multi(const MultiRedItem* items, int n_items, int n_ctas, cudaStream_t st)
{
    void* args[] = {(void*)&items, (void*)&n_items};
    return launch_pdl((const void*)fwd_reduce_multi_kernel, dim3(n_ctas), dim3(RED_OUT * 32), 0, st, args);
}

int fwd_reduce_blocks(int n_out) { return (n_out + RED_OUT - 1) / RED_OUT; }

cudaError_t launch_fwd_reduce(const OpDesc& op, const ReduceArgs& a, cudaStream_t st)
{
    dim3 grid((a.n_out + RED_OUT - 1) / RED_OUT);
    void* args[] = {(void*)&op, (void*)&a};
    return launch_pdl((const void*)fwd_reduce_kernel, grid, dim3(RED_OUT * 32), 0, st, args);
}

}  // namespace nfm
