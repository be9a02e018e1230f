// Minibatch adjoint g = A_B^H r on CUDA cores, optionally fused with the SPGM
// gradient step and the complex soft-threshold (Eq. 5 with the Eq. 6 gradient):
//
//     s_n <- prox( s_n - (eta/B) g_n ),  prox(z) = z max(0, 1 - alpha/|z|) / (1 + eta lambda w2)
//
// (alpha = eta lambda w1; w2 = 0 is the paper's l1 prox).
//
// One CTA = one 8x4x4 voxel tile, 128 threads: two voxels per thread (z layers
// lz and lz+2) and the minibatch pairs split by parity between two thread
// halves, combined in a fixed order at the end.  Each voxel is owned by one
// CTA, so no reduction across CTAs is needed.  For a pair and a voxel the sum over the K
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

// Phasors of one (pair, voxel): a = amp e^{+j 2 pi f0 D/c}, z, Z.
struct AdjPhasors {
    float2 a, z, Z;
};

template <int K1>
__device__ __forceinline__ AdjPhasors adj_phasors(const PairTile& P, const VoxelOffset& o, const PhaseConsts& ph)
{
    const PVGeom G = pair_voxel(P, o, ph);
    AdjPhasors f;
    const float2 c = cis_turns_sfu(G.th0);
    f.a = make_float2(G.amp * c.x, G.amp * c.y);
    f.z = cis_turns(G.dth);
    f.Z = K1 > 1 ? cis_turns_sfu(G.dth2) : make_float2(1.f, 0.f);
    return f;
}

// sum_k z^k r_k for one voxel: K1 inner Horner chains of K2 terms, then Horner in Z.
template <int K1>
__device__ __forceinline__ float2 adj_poly(const float2* __restrict__ rj, const AdjPhasors& f0, const AdjPhasors& f1,
                                           float2& out1)
{
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
            const float2 a0 = h0[q], a1 = h1[q];
            h0[q] = make_float2(fmaf(a0.x, f0.z.x, fmaf(-a0.y, f0.z.y, rv.x)),
                                fmaf(a0.x, f0.z.y, fmaf(a0.y, f0.z.x, rv.y)));
            h1[q] = make_float2(fmaf(a1.x, f1.z.x, fmaf(-a1.y, f1.z.y, rv.x)),
                                fmaf(a1.x, f1.z.y, fmaf(a1.y, f1.z.x, rv.y)));
        }
    }
    float2 S0 = h0[K1 - 1], S1 = h1[K1 - 1];
#pragma unroll
    for (int q = K1 - 2; q >= 0; --q) {
        S0 = cmul(S0, f0.Z);
        S0.x += h0[q].x;
        S0.y += h0[q].y;
        S1 = cmul(S1, f1.Z);
        S1.x += h1[q].x;
        S1.y += h1[q].y;
    }
    out1 = cmul(f1.a, S1);
    return cmul(f0.a, S0);
}

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
    const int half = tid / 64;                       // pair parity this thread handles
    const int lt = tid % 64;
    const int lx = lt % TILE_X;
    const int ly = (lt / TILE_X) % TILE_Y;
    const int lz = lt / (TILE_X * TILE_Y);           // 0 or 1; second voxel at lz + 2
    const VoxelOffset o0 = voxel_offset(op.g, lx, ly, lz);
    const VoxelOffset o1 = voxel_offset(op.g, lx, ly, lz + 2);
    constexpr int KB = K1 * K2;

    float2 g0 = make_float2(0.f, 0.f), g1 = make_float2(0.f, 0.f);
    pdl_wait();                              // r comes from the previous kernel

    for (int c0 = 0; c0 < a.n_pairs; c0 += a.pchunk) {
        const int nc = min(a.pchunk, a.n_pairs - c0);
        __syncthreads();
        for (int e = tid; e < nc * KB; e += ADJ_THREADS) {
            const int j = e / KB;
            const int kk = e - j * KB;
            float2 v = make_float2(0.f, 0.f);
            if (kk < op.K) {
                v = a.r[(size_t)(c0 + j) * op.K + kk];
                if (op.pulse) v = cmul_conj(v, op.pulse[kk]);   // conj(p_k) r
            }
            const int k1 = kk / K2, k2 = kk - (kk / K2) * K2;
            rs[(j * K2 + k2) * K1 + k1] = v;
        }
        for (int j = tid; j < nc; j += ADJ_THREADS) pt[j] = load_pair_tile(op, a.pairs[c0 + j], tile);
        __syncthreads();

        // software pipeline: phasors of the next pair are computed while the
        // Horner chains of the current pair run (independent instructions)
        int j = half;
        if (j < nc) {
            AdjPhasors f0 = adj_phasors<K1>(pt[j], o0, op.ph);
            AdjPhasors f1 = adj_phasors<K1>(pt[j], o1, op.ph);
            for (; j < nc; j += 2) {
                const int jn = min(j + 2, nc - 1);
                const AdjPhasors n0 = adj_phasors<K1>(pt[jn], o0, op.ph);
                const AdjPhasors n1 = adj_phasors<K1>(pt[jn], o1, op.ph);
                float2 t1;
                const float2 t0 = adj_poly<K1>(rs + j * KB, f0, f1, t1);
                g0.x += t0.x;
                g0.y += t0.y;
                g1.x += t1.x;
                g1.y += t1.y;
                f0 = n0;
                f1 = n1;
            }
        }
    }

    // combine the two pair halves in a fixed order, then the epilogue
    pdl_launch_dependents();
    __syncthreads();
    float2* comb = reinterpret_cast<float2*>(smem);   // [64][2]
    if (half == 1) {
        comb[2 * lt] = g0;
        comb[2 * lt + 1] = g1;
    }
    __syncthreads();
    if (half == 1) return;
    {
        const float2 b0 = comb[2 * lt], b1 = comb[2 * lt + 1];
        g0.x += b0.x;
        g0.y += b0.y;
        g1.x += b1.x;
        g1.y += b1.y;
    }
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
                float sc = (1.0f - a.alpha / mag) * a.shrink;
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
    size_t b = (size_t)pchunk * K2 * K1 * sizeof(float2) + (size_t)pchunk * sizeof(PairTile);
    size_t comb = 128 * sizeof(float2);
    return b > comb ? b : comb;
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
    const void* fn = adj_kernel_ptr(op.K1);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&op, (void*)&a};
    return launch_pdl(fn, dim3(op.g.n_tiles), dim3(ADJ_THREADS), smem, st, args);
}

}  // namespace nfm
