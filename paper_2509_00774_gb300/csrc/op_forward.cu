// Minibatch forward operator y = A_B s on CUDA cores (Eq. 2 rows of a pair list).
//
// Work split: blockIdx.x = group of FWD_PC pairs, blockIdx.y = chunk of voxel
// tiles (a contiguous tile range).  Each CTA writes a partial spectrum
// [FWD_PC][K] for its chunk; fwd_reduce_kernel sums the chunks in a fixed
// order, so the result does not depend on scheduling.
//
// Per tile the CTA
//  1. stages s for the tile's voxels and the Pc (pair, tile) constants,
//  2. for every (voxel, pair) builds the block start values
//        U[k1] = amp s exp(-j 2 pi (f0 + k1 K2 df) D / c)      (k1 < K1)
//     and the fine step w = exp(-j 2 pi df D / c) in shared memory,
//  3. thread (pair, k1, vs) walks its voxels two at a time and accumulates
//     the K2 frequencies of block k1 with the recurrence t <- t w (6 FP32
//     lane-instructions per (row, voxel) element).
#include "nfm_kernels.cuh"

namespace nfm {

template <int K1>
__global__ void __launch_bounds__(256, 3) fwd_partial_kernel(OpDesc op, FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int PC = FWD_PC;
    const int VS = a.VS;
    const int nt = blockDim.x;
    const int tid = threadIdx.x;
    const int group = blockIdx.x;
    const int chunk = blockIdx.y;

    float2* U = reinterpret_cast<float2*>(smem);          // [TILE_V][K1][PC]
    float2* Wf = U + TILE_V * PC * K1;                    // [TILE_V][PC]
    float2* s_t = Wf + TILE_V * PC;                       // [TILE_V]
    PairTile* pt = reinterpret_cast<PairTile*>(s_t + TILE_V);   // [PC]
    int* pair_s = reinterpret_cast<int*>(pt + PC);        // [PC]

    // main-loop role: pair fastest so a warp reads 32 consecutive U entries
    const int p = tid % PC;
    const int k1 = (tid / PC) % K1;
    const int vs = tid / (PC * K1);

    float2 acc[K2];
#pragma unroll
    for (int i = 0; i < K2; ++i) acc[i] = make_float2(0.f, 0.f);

    const int t_begin = chunk * a.tiles_base + min(chunk, a.tiles_rem);
    const int t_end = t_begin + a.tiles_base + (chunk < a.tiles_rem ? 1 : 0);

    if (tid < PC) {
        int slot = group * PC + tid;
        pair_s[tid] = slot < a.n_pairs ? a.pairs[slot] : -1;
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
        if (tid < PC) {
            int pair = pair_s[tid];
            pt[tid] = load_pair_tile(op, pair < 0 ? 0 : pair, tile);
        }
        __syncthreads();
        // staging: item = v * PC + i
#pragma unroll 2
        for (int item = tid; item < TILE_V * PC; item += nt) {
            const int i = item % PC;
            const int v = item / PC;
            float2* Up = U + v * (K1 * PC) + i;
            if (pair_s[i] < 0) {
#pragma unroll
                for (int j = 0; j < K1; ++j) Up[j * PC] = make_float2(0.f, 0.f);
                Wf[item] = make_float2(1.f, 0.f);
                continue;
            }
            const int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y);
            const float2 sv = s_t[v];
            const VoxelOffset o = voxel_offset(op.g, lx, ly, lz);
            const PVGeom gv = pair_voxel(pt[i], o, op.ph);
            const float2 c0 = cis_turns(gv.th0);
            const float2 cw = cis_turns(gv.dth);
            float2 u = cmul_conj(make_float2(gv.amp * sv.x, gv.amp * sv.y), c0);
            Up[0] = u;
            if (K1 > 1) {
                const float2 cW = cis_turns(gv.dth2);
                const float2 Wc = make_float2(cW.x, -cW.y);
#pragma unroll
                for (int j = 1; j < K1; ++j) {
                    u = cmul(u, Wc);
                    Up[j * PC] = u;
                }
            }
            Wf[item] = make_float2(cw.x, -cw.y);
        }
        __syncthreads();
        // main loop: two voxels per step for two independent recurrences
        if (vs < VS) {
            int v = vs;
            for (; v + VS < TILE_V; v += 2 * VS) {
                float2 t0 = U[v * (K1 * PC) + k1 * PC + p];
                float2 w0 = Wf[v * PC + p];
                float2 t1 = U[(v + VS) * (K1 * PC) + k1 * PC + p];
                float2 w1 = Wf[(v + VS) * PC + p];
#pragma unroll
                for (int j = 0; j < K2; ++j) {
                    acc[j].x += t0.x + t1.x;
                    acc[j].y += t0.y + t1.y;
                    if (j + 1 < K2) {
                        t0 = cmul(t0, w0);
                        t1 = cmul(t1, w1);
                    }
                }
            }
            if (v < TILE_V) {
                float2 t0 = U[v * (K1 * PC) + k1 * PC + p];
                float2 w0 = Wf[v * PC + p];
#pragma unroll
                for (int j = 0; j < K2; ++j) {
                    acc[j].x += t0.x;
                    acc[j].y += t0.y;
                    if (j + 1 < K2) t0 = cmul(t0, w0);
                }
            }
        }
    }

    // reduce the VS voxel subsets in a fixed order, then write the partial
    __syncthreads();
    float2* red = reinterpret_cast<float2*>(smem);        // [VS][PC][K1*K2]
    constexpr int KB = K1 * K2;
    if (vs < VS) {
#pragma unroll
        for (int j = 0; j < K2; ++j) red[((vs * PC + p) * K1 + k1) * K2 + j] = acc[j];
    }
    __syncthreads();
    for (int o = tid; o < PC * KB; o += nt) {
        int i = o / KB;
        int kk = o - i * KB;
        int slot = group * PC + i;
        if (kk >= op.K || slot >= a.n_pairs) continue;
        float2 sum = red[i * KB + kk];
        for (int u = 1; u < VS; ++u) {
            float2 x = red[(u * PC + i) * KB + kk];
            sum.x += x.x;
            sum.y += x.y;
        }
        a.partial[((size_t)chunk * a.n_slots + slot) * op.K + kk] = sum;
    }
}

size_t fwd_smem_bytes(int K1, int nt)
{
    const int Pc = FWD_PC;
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
__global__ void __launch_bounds__(1024) fwd_reduce_kernel(OpDesc op, ReduceArgs a)
{
    __shared__ float2 red[32][33];
    const int o = blockIdx.x * 32 + threadIdx.x;
    const size_t stride = (size_t)a.n_slots * op.K;
    float2 s = make_float2(0.f, 0.f);
    if (o < a.n_out) {
        // chunk lane y sums chunks y, y+32, ... (four loads in flight, fixed order)
        int c = threadIdx.y;
        for (; c + 96 < a.n_chunks; c += 128) {
            float2 x0 = a.partial[(size_t)c * stride + o];
            float2 x1 = a.partial[(size_t)(c + 32) * stride + o];
            float2 x2 = a.partial[(size_t)(c + 64) * stride + o];
            float2 x3 = a.partial[(size_t)(c + 96) * stride + o];
            s.x += ((x0.x + x1.x) + (x2.x + x3.x));
            s.y += ((x0.y + x1.y) + (x2.y + x3.y));
        }
        for (; c < a.n_chunks; c += 32) {
            float2 x = a.partial[(size_t)c * stride + o];
            s.x += x.x;
            s.y += x.y;
        }
    }
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && o < a.n_out) {
        float2 t = red[0][threadIdx.x];
#pragma unroll
        for (int y = 1; y < 32; ++y) {
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
    dim3 block(32, 32);
    dim3 grid((a.n_out + 31) / 32);
    fwd_reduce_kernel<<<grid, block, 0, st>>>(op, a);
    return cudaGetLastError();
}

}  // namespace nfm
