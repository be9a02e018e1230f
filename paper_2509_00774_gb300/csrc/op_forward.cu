// Minibatch forward operator y = A_B s on CUDA cores (Eq. 2 rows of a pair list).
//
// Work split: blockIdx.x = group of Pc pairs, blockIdx.y = chunk of voxel
// tiles (a contiguous tile range).  Each CTA writes a partial spectrum
// [Pc][K] for its chunk; nfm_fwd_reduce sums the chunks in a fixed order, so
// the result does not depend on scheduling.
//
// Per tile the CTA
//  1. stages s for the tile's voxels and the Pc (pair, tile) constants,
//  2. for every (voxel, pair) builds the block start values
//        U[k1] = amp s exp(-j 2 pi (f0 + k1 K2 df) D / c)      (k1 < K1)
//     and the fine step w = exp(-j 2 pi df D / c) in shared memory,
//  3. thread (k1, pair, vs) walks its voxels and accumulates the K2
//     frequencies of block k1 with the recurrence t <- t w (6 FP32
//     lane-instructions per (row, voxel) element).
#include "nfm_kernels.cuh"

namespace nfm {

template <int K1>
__global__ void __launch_bounds__(256) fwd_partial_kernel(OpDesc op, FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int Pc = a.Pc;
    const int VS = a.VS;
    const int nt = blockDim.x;
    const int tid = threadIdx.x;
    const int group = blockIdx.x;
    const int chunk = blockIdx.y;

    float2* U = reinterpret_cast<float2*>(smem);          // [TILE_V][Pc][K1]
    float2* Wf = U + TILE_V * Pc * K1;                    // [TILE_V][Pc]
    float2* s_t = Wf + TILE_V * Pc;                       // [TILE_V]
    PairTile* pt = reinterpret_cast<PairTile*>(s_t + TILE_V);   // [Pc]
    int* pair_s = reinterpret_cast<int*>(pt + Pc);        // [Pc]

    const int k1 = tid % K1;
    const int p = (tid / K1) % Pc;
    const int vs = tid / (K1 * Pc);

    float2 acc[K2];
#pragma unroll
    for (int i = 0; i < K2; ++i) acc[i] = make_float2(0.f, 0.f);

    const int t_begin = chunk * a.tiles_base + min(chunk, a.tiles_rem);
    const int t_end = t_begin + a.tiles_base + (chunk < a.tiles_rem ? 1 : 0);

    for (int i = tid; i < Pc; i += nt) {
        int slot = group * Pc + i;
        pair_s[i] = slot < a.n_pairs ? a.pairs[slot] : -1;
    }

    for (int tile = t_begin; tile < t_end; ++tile) {
        int tx, ty, tz;
        tile_coords(op.g, tile, tx, ty, tz);
        __syncthreads();   // previous tile fully consumed; pair_s visible
        for (int v = tid; v < TILE_V; v += nt) {
            int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y);
            int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
            float2 sv = make_float2(0.f, 0.f);
            if (ix < op.g.nx && iy < op.g.ny && iz < op.g.nz)
                sv = a.s[((size_t)iz * op.g.ny + iy) * op.g.nx + ix];
            s_t[v] = sv;
        }
        for (int i = tid; i < Pc; i += nt) {
            int pair = pair_s[i];
            pt[i] = load_pair_tile(op, pair < 0 ? 0 : pair, tile);
        }
        __syncthreads();
        for (int item = tid; item < TILE_V * Pc; item += nt) {
            int i = item % Pc;
            int v = item / Pc;
            float2* Up = U + (v * Pc + i) * K1;
            int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y);
            float2 sv = s_t[v];
            if (pair_s[i] < 0) sv = make_float2(0.f, 0.f);
            VoxelOffset o = voxel_offset(op.g, lx, ly, lz);
            PVGeom gv = pair_voxel(pt[i], o, op.ph);
            float2 c0 = cis_turns(gv.th0);
            float2 cw = cis_turns(gv.dth);
            float2 cW = cis_turns(gv.dth2);
            float2 u = cmul_conj(make_float2(gv.amp * sv.x, gv.amp * sv.y), c0);
            float2 Wc = make_float2(cW.x, -cW.y);
            Up[0] = u;
#pragma unroll
            for (int j = 1; j < K1; ++j) {
                u = cmul(u, Wc);
                Up[j] = u;
            }
            Wf[v * Pc + i] = make_float2(cw.x, -cw.y);
        }
        __syncthreads();
        if (vs < VS) {
            for (int v = vs; v < TILE_V; v += VS) {
                float2 t = U[(v * Pc + p) * K1 + k1];
                float2 w = Wf[v * Pc + p];
#pragma unroll
                for (int j = 0; j < K2; ++j) {
                    acc[j].x += t.x;
                    acc[j].y += t.y;
                    if (j + 1 < K2) t = cmul(t, w);
                }
            }
        }
    }

    // reduce the VS voxel subsets in a fixed order, then write the partial
    __syncthreads();
    float2* red = reinterpret_cast<float2*>(smem);        // [VS][Pc][K1*K2]
    constexpr int KB = K1 * K2;
    if (vs < VS) {
#pragma unroll
        for (int j = 0; j < K2; ++j) red[((vs * Pc + p) * K1 + k1) * K2 + j] = acc[j];
    }
    __syncthreads();
    for (int o = tid; o < Pc * KB; o += nt) {
        int i = o / KB;
        int kk = o - i * KB;
        int slot = group * Pc + i;
        if (kk >= op.K || slot >= a.n_pairs) continue;
        float2 sum = red[i * KB + kk];
        for (int u = 1; u < VS; ++u) {
            float2 x = red[(u * Pc + i) * KB + kk];
            sum.x += x.x;
            sum.y += x.y;
        }
        a.partial[((size_t)chunk * a.n_slots + slot) * op.K + kk] = sum;
    }
}

size_t fwd_smem_bytes(int K1, int Pc, int nt)
{
    size_t stage = (size_t)TILE_V * Pc * (K1 + 1) * sizeof(float2) + TILE_V * sizeof(float2) +
                   (size_t)Pc * sizeof(PairTile) + (size_t)Pc * sizeof(int);
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
    switch (op.K1) {
    case 1: fwd_partial_kernel<1><<<grid, nt, smem, st>>>(op, a); break;
    case 2: fwd_partial_kernel<2><<<grid, nt, smem, st>>>(op, a); break;
    case 3: fwd_partial_kernel<3><<<grid, nt, smem, st>>>(op, a); break;
    case 4: fwd_partial_kernel<4><<<grid, nt, smem, st>>>(op, a); break;
    case 5: fwd_partial_kernel<5><<<grid, nt, smem, st>>>(op, a); break;
    case 6: fwd_partial_kernel<6><<<grid, nt, smem, st>>>(op, a); break;
    case 7: fwd_partial_kernel<7><<<grid, nt, smem, st>>>(op, a); break;
    case 8: fwd_partial_kernel<8><<<grid, nt, smem, st>>>(op, a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Sum the chunk partials in chunk order (fixed), apply p(f_k), and optionally
// subtract the observed rows: out[slot*K + k] = p_k sum_c partial[c][slot][k] - y[pair*K + k].
__global__ void __launch_bounds__(256) fwd_reduce_kernel(OpDesc op, ReduceArgs a)
{
    __shared__ float2 red[8][33];
    const int o = blockIdx.x * 32 + threadIdx.x;
    float2 s = make_float2(0.f, 0.f);
    if (o < a.n_out) {
        for (int c = threadIdx.y; c < a.n_chunks; c += 8) {
            float2 x = a.partial[(size_t)c * a.n_slots * op.K + o];
            s.x += x.x;
            s.y += x.y;
        }
    }
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && o < a.n_out) {
        float2 t = red[0][threadIdx.x];
#pragma unroll
        for (int y = 1; y < 8; ++y) {
            t.x += red[y][threadIdx.x].x;
            t.y += red[y][threadIdx.x].y;
        }
        int k = o % op.K;
        if (op.pulse) t = cmul(op.pulse[k], t);
        if (a.y_obs) {
            int pair = a.pairs[o / op.K];
            if (pair < 0 || pair >= op.P) {
                atomicOr(op.err, ERRF_PAIR);
                pair = 0;
            }
            float2 yo = a.y_obs[(size_t)pair * op.K + k];
            t.x -= yo.x;
            t.y -= yo.y;
        }
        a.out[o] = t;
    }
}

cudaError_t launch_fwd_reduce(const OpDesc& op, const ReduceArgs& a, cudaStream_t st)
{
    dim3 block(32, 8);
    dim3 grid((a.n_out + 31) / 32);
    fwd_reduce_kernel<<<grid, block, 0, st>>>(op, a);
    return cudaGetLastError();
}

}  // namespace nfm
