// Minibatch adjoint g = A_B^H r on CUDA cores, optionally fused with the SPGM
// gradient step and the complex soft-threshold (Eq. 5 with the Eq. 6 gradient):
//
//     s_n <- prox_alpha( s_n - (eta/B) g_n ),  prox(z) = z max(0, 1 - alpha/|z|).
//
// One CTA = one 8x4x4 voxel tile, 64 threads, two voxels per thread (z layers
// lz and lz+2), so each voxel is owned by exactly one thread and no reduction
// across CTAs is needed.  For a pair and a voxel the sum over the K
// frequencies is a polynomial in z = exp(+j 2 pi df D/c):
//
//     sum_k conj(A_k) r_k = amp e^{+j 2 pi f0 D/c} sum_k1 Z^k1 sum_k2 z^k2 r[k1 K2 + k2],
//     Z = z^K2 = exp(+j 2 pi K2 df D/c),
//
// evaluated by Horner's rule: the K1 inner polynomials (K2 terms each, 4 FP32
// FMAs per term) run as independent chains, then one outer Horner pass in Z.
// r is staged in shared memory as [pair][k2][k1] so the K1 values a step
// needs are contiguous.
#include "nfm_kernels.cuh"

namespace nfm {

template <int K1>
__global__ void __launch_bounds__(ADJ_THREADS) adj_kernel(OpDesc op, AdjArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float2* rs = reinterpret_cast<float2*>(smem);                        // [pchunk][K2][K1]
    PairTile* pt = reinterpret_cast<PairTile*>(rs + a.pchunk * K2 * K1);  // [pchunk]

    const int tile = blockIdx.x;
    int tx, ty, tz;
    tile_coords(op.g, tile, tx, ty, tz);
    const int tid = threadIdx.x;
    const int lx = tid % TILE_X;
    const int ly = (tid / TILE_X) % TILE_Y;
    const int lz = tid / (TILE_X * TILE_Y);          // 0 or 1; second voxel at lz + 2
    const VoxelOffset o0 = voxel_offset(op.g, lx, ly, lz);
    const VoxelOffset o1 = voxel_offset(op.g, lx, ly, lz + 2);
    constexpr int KB = K1 * K2;

    float2 g0 = make_float2(0.f, 0.f), g1 = make_float2(0.f, 0.f);

    for (int c0 = 0; c0 < a.n_pairs; c0 += a.pchunk) {
        const int nc = min(a.pchunk, a.n_pairs - c0);
        __syncthreads();
        for (int e = tid; e < nc * KB; e += ADJ_THREADS) {
            int j = e / KB;
            int kk = e - j * KB;
            float2 v = make_float2(0.f, 0.f);
            if (kk < op.K) {
                v = a.r[(size_t)(c0 + j) * op.K + kk];
                if (op.pulse) v = cmul_conj(v, op.pulse[kk]);   // conj(p_k) r
            }
            int k1 = kk / K2, k2 = kk - (kk / K2) * K2;
            rs[(j * K2 + k2) * K1 + k1] = v;
        }
        for (int j = tid; j < nc; j += ADJ_THREADS) pt[j] = load_pair_tile(op, a.pairs[c0 + j], tile);
        __syncthreads();

        for (int j = 0; j < nc; ++j) {
            const PairTile P = pt[j];
            const PVGeom G0 = pair_voxel(P, o0, op.ph);
            const PVGeom G1 = pair_voxel(P, o1, op.ph);
            const float2 z0 = cis_turns(G0.dth), z1 = cis_turns(G1.dth);
            const float2* rj = rs + j * KB;
            float2 h0[K1], h1[K1];
#pragma unroll
            for (int q = 0; q < K1; ++q) {
                h0[q] = rj[(K2 - 1) * K1 + q];
                h1[q] = h0[q];
            }
#pragma unroll
            for (int k2 = K2 - 2; k2 >= 0; --k2) {
#pragma unroll
                for (int q = 0; q < K1; ++q) {
                    const float2 rv = rj[k2 * K1 + q];
                    float2 a0 = h0[q], a1 = h1[q];
                    h0[q] = make_float2(fmaf(a0.x, z0.x, fmaf(-a0.y, z0.y, rv.x)),
                                        fmaf(a0.x, z0.y, fmaf(a0.y, z0.x, rv.y)));
                    h1[q] = make_float2(fmaf(a1.x, z1.x, fmaf(-a1.y, z1.y, rv.x)),
                                        fmaf(a1.x, z1.y, fmaf(a1.y, z1.x, rv.y)));
                }
            }
            float2 S0 = h0[K1 - 1], S1 = h1[K1 - 1];
            if (K1 > 1) {
                const float2 Z0 = cis_turns(G0.dth2), Z1 = cis_turns(G1.dth2);
#pragma unroll
                for (int q = K1 - 2; q >= 0; --q) {
                    S0 = cmul(S0, Z0);
                    S0.x += h0[q].x;
                    S0.y += h0[q].y;
                    S1 = cmul(S1, Z1);
                    S1.x += h1[q].x;
                    S1.y += h1[q].y;
                }
            }
            const float2 c00 = cis_turns(G0.th0), c01 = cis_turns(G1.th0);
            const float2 t0 = cmul(c00, S0), t1 = cmul(c01, S1);
            g0.x = fmaf(G0.amp, t0.x, g0.x);
            g0.y = fmaf(G0.amp, t0.y, g0.y);
            g1.x = fmaf(G1.amp, t1.x, g1.x);
            g1.y = fmaf(G1.amp, t1.y, g1.y);
        }
    }

    // epilogue: plain adjoint, or gradient step + prox in place
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz + 2 * h;
        if (ix >= op.g.nx || iy >= op.g.ny || iz >= op.g.nz) continue;
        const size_t n = ((size_t)iz * op.g.ny + iy) * op.g.nx + ix;
        const float2 g = h ? g1 : g0;
        if (a.s) {
            float2 sv = a.s[n];
            float zr = fmaf(-a.step, g.x, sv.x);
            float zi = fmaf(-a.step, g.y, sv.y);
            float mag = sqrtf(zr * zr + zi * zi);
            float2 out = make_float2(0.f, 0.f);
            if (mag > a.alpha) {
                float sc = 1.0f - a.alpha / mag;
                out = make_float2(zr * sc, zi * sc);
            }
            a.s[n] = out;
        } else {
            a.g_out[n] = g;
        }
    }
}

size_t adj_smem_bytes(int K1, int pchunk)
{
    return (size_t)pchunk * K2 * K1 * sizeof(float2) + (size_t)pchunk * sizeof(PairTile);
}

const void* adj_kernel_ptr(int K1)
{
    switch (K1) {
    case 1: return (const void*)adj_kernel<1>;
    case 2: return (const void*)adj_kernel<2>;
    case 3: return (const void*)adj_kernel<3>;
    case 4: return (const void*)adj_kernel<4>;
    case 5: return (const void*)adj_kernel<5>;
    case 6: return (const void*)adj_kernel<6>;
    case 7: return (const void*)adj_kernel<7>;
    case 8: return (const void*)adj_kernel<8>;
    default: return nullptr;
    }
}

cudaError_t launch_adjoint(const OpDesc& op, const AdjArgs& a, size_t smem, cudaStream_t st)
{
    dim3 grid(op.g.n_tiles);
    switch (op.K1) {
    case 1: adj_kernel<1><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    case 2: adj_kernel<2><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    case 3: adj_kernel<3><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    case 4: adj_kernel<4><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    case 5: adj_kernel<5><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    case 6: adj_kernel<6><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    case 7: adj_kernel<7><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    case 8: adj_kernel<8><<<grid, ADJ_THREADS, smem, st>>>(op, a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace nfm
