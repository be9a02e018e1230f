// Tensor-core (tcgen05) form of the minibatch adjoint g = A_B^H r, optionally
// fused with the SPGM gradient step and prox (Eq. 5 with the Eq. 6 gradient).
//
// For one pair and the 128 voxels v of an 8x4x4 tile, with z_v = exp(+j 2 pi df D_v/c),
//
//     H[v, k1] = sum_{k2 < 16} z_v^k2 r[k1*16 + k2]             (complex)
//
// is a real GEMM D = A B^T with M = 128 (voxels), K = 32 ((k2, re/im)) and
// N = 16 (rows (k1, re/im); 2 K1 of them used):
//     A[v, (k2, 0)] = Re z^k2,  A[v, (k2, 1)] = Im z^k2,
//     B[(k1, 0), (k2, 0)] = Re r,  B[(k1, 0), (k2, 1)] = -Im r,
//     B[(k1, 1), (k2, 0)] = Im r,  B[(k1, 1), (k2, 1)] =  Re r.
// Each FP32 operand x is split as x = hi + lo in BF16 (or FP16, r scaled per
// pair by a power of two) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// accumulates in FP32 in tensor memory.  The rest of the sum over k1 is the
// outer Horner pass of the CUDA-core adjoint: g_v += a_v sum_k1 Z_v^k1 H[v, k1].
//
// Per CTA (128 threads = 128 voxels, one tile): thread v generates its A row
// for pair q into one of two shared buffers while the tensor core runs pair
// q-1; the result of pair q-2 is read from one of two TMEM accumulators.
// Operands use the no-swizzle K-major layout: 8-row x 16-byte core matrices,
// core matrices along K 128 B apart (LBO), along M/N 256 B apart (SBO).
#include "nfm_kernels.cuh"
#include "tc_ptx.cuh"

namespace nfm {

namespace {

using namespace tc;

constexpr int TC_M = 128;
constexpr int TC_N = 16;
constexpr int TC_KSTEP_BYTES_A = TC_M * 16 * 2;    // 4096: one K step (16 elements) of A
constexpr int TC_KSTEP_BYTES_B = TC_N * 16 * 2;    // 512
constexpr int TC_B_PAIR_BYTES = 2 * 2 * TC_KSTEP_BYTES_B;   // [split][kstep] = 2048

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (or F16), both K-major, M = 128, N = 16.
template <bool F16>
__host__ __device__ constexpr uint32_t tc_idesc()
{
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(TC_N >> 3) << 17) |
           ((uint32_t)(TC_M >> 4) << 24);
}

}  // namespace

// B operand of every minibatch pair: [n_pairs][split][kstep][16 rows x 16 K] in the
// K-major core-matrix layout, and the per-pair power-of-two scale (FP16 only).
template <bool F16>
__global__ void __launch_bounds__(128) adj_tc_prep_kernel(OpDesc op, const float2* r, int n_pairs,
                                                          unsigned char* bmat, float* inv_scale)
{
    const int j = blockIdx.x;
    const int k = threadIdx.x;             // frequency index, k < 128
    pdl_wait();
    float2 v = make_float2(0.f, 0.f);
    if (k < op.K && j < n_pairs) {
        v = r[(size_t)j * op.K + k];
        if (op.pulse) v = cmul_conj(v, op.pulse[k]);
    }
    float scale = 1.0f, inv = 1.0f;
    if (F16) {
        __shared__ float wmax[4];
        float m = fmaxf(fabsf(v.x), fabsf(v.y));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((k & 31) == 0) wmax[k >> 5] = m;
        __syncthreads();
        m = fmaxf(fmaxf(wmax[0], wmax[1]), fmaxf(wmax[2], wmax[3]));
        if (m > 0.f) {
            int e;
            frexpf(m, &e);                  // m = f 2^e, f in [0.5, 1)
            scale = ldexpf(1.0f, -e);       // |scaled| < 1
            inv = ldexpf(1.0f, e);
        }
    }
    v.x *= scale;
    v.y *= scale;
    unsigned char* bp = bmat + (size_t)j * TC_B_PAIR_BYTES;
    const int k1 = k / K2, k2 = k % K2;
    const int s = k2 / 8, kk = 2 * (k2 % 8);
    if (k1 < MAX_K1) {
        uint32_t h0, l0, h1, l1;
        split2<F16>(v.x, -v.y, h0, l0);     // row (k1, re): ( Re r, -Im r)
        split2<F16>(v.y, v.x, h1, l1);      // row (k1, im): ( Im r,  Re r)
        const bool used = k1 < op.K1;
        const int row0 = 2 * k1, row1 = 2 * k1 + 1;
        if (row1 < TC_N) {
            *reinterpret_cast<uint32_t*>(bp + 0 * 2 * TC_KSTEP_BYTES_B + s * TC_KSTEP_BYTES_B + kmaj_off(row0, kk)) = used ? h0 : 0u;
            *reinterpret_cast<uint32_t*>(bp + 0 * 2 * TC_KSTEP_BYTES_B + s * TC_KSTEP_BYTES_B + kmaj_off(row1, kk)) = used ? h1 : 0u;
            *reinterpret_cast<uint32_t*>(bp + 1 * 2 * TC_KSTEP_BYTES_B + s * TC_KSTEP_BYTES_B + kmaj_off(row0, kk)) = used ? l0 : 0u;
            *reinterpret_cast<uint32_t*>(bp + 1 * 2 * TC_KSTEP_BYTES_B + s * TC_KSTEP_BYTES_B + kmaj_off(row1, kk)) = used ? l1 : 0u;
        }
    }
    if (k == 0) inv_scale[j] = inv;
    pdl_launch_dependents();
}

template <int K1, bool F16>
__global__ void __launch_bounds__(128) adj_tc_kernel(OpDesc op, AdjArgs a, const unsigned char* bmat,
                                                     const float* inv_scale)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // A: [buf 2][split 2][kstep 2][4096]  B: [pchunk][2048]  then pair tiles, scales, barriers
    unsigned char* As = smem;
    unsigned char* Bs = As + 2 * 2 * 2 * TC_KSTEP_BYTES_A;
    PairTile* pt = reinterpret_cast<PairTile*>(Bs + (size_t)a.pchunk * TC_B_PAIR_BYTES);
    float* sc = reinterpret_cast<float*>(pt + a.pchunk);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sc + ((a.pchunk + 1) & ~1));
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);

    const int tile = blockIdx.x;
    int tx, ty, tz;
    tile_coords(op.g, tile, tx, ty, tz);
    const int v = threadIdx.x;             // voxel = TMEM lane = A row
    const int warp = v / 32;
    const int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y);
    const VoxelOffset o = voxel_offset(op.g, lx, ly, lz);
    constexpr uint32_t IDESC = tc_idesc<F16>();

    if (warp == 0) {
        tmem_alloc(tslot, 32);
        tmem_relinquish();
    }
    if (v == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    bool ok = true;

    float2 g = make_float2(0.f, 0.f);
    // pending pairs (ring of two, slot = pair & 1): phasor a, block step Z and 1/scale
    float2 pa0 = make_float2(0.f, 0.f), pa1 = pa0, pZ0 = pa0, pZ1 = pa0;
    float pinv0 = 0.f, pinv1 = 0.f;
    int issued = 0;                        // pairs whose MMAs are issued (chunk granularity)
    int done = 0;                          // pairs whose result has been read back
    int committed = 0;                     // pairs whose MMAs were actually committed (same in every thread)
    const bool issue = !(op.hooks & HOOK_TC_SKIP_ISSUE);

    auto finish = [&](int q) {             // read TMEM of pair q and add its contribution
        if (!ok) return;                   // after a timeout: no TMEM reads (ok is uniform over the CTA)
        const int buf = q & 1;
        // uniform outcome; on a timeout every committed pair from q on gets one more bounded wait so that
        // no MMA is in flight when TMEM is released, no further MMA is issued, and the output is left unwritten
        if (!__syncthreads_and(mbar_wait(&bar[buf], (uint32_t)((q >> 1) & 1), op.wait_ns))) {
            for (int qq = q; qq < committed; ++qq) mbar_wait(&bar[qq & 1], (uint32_t)((qq >> 1) & 1), op.wait_ns);
            ok = false;
            return;
        }
        tc_fence_after();
        float h[16];
        tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * TC_N), h);
        const float2 Zq = buf ? pZ1 : pZ0, aq = buf ? pa1 : pa0;
        const float iq = buf ? pinv1 : pinv0;
        float2 S = make_float2(h[2 * (K1 - 1)], h[2 * (K1 - 1) + 1]);
#pragma unroll
        for (int k1 = K1 - 2; k1 >= 0; --k1) {
            S = cmul(S, Zq);
            S.x += h[2 * k1];
            S.y += h[2 * k1 + 1];
        }
        const float2 t = cmul(aq, S);
        g.x = fmaf(iq, t.x, g.x);
        g.y = fmaf(iq, t.y, g.y);
    };

    auto finish_until = [&](int upto) {
        while (done < upto) finish(done++);
    };

    pdl_wait();                            // r (through bmat) comes from the previous kernels
    for (int c0 = 0; c0 < a.n_pairs; c0 += a.pchunk) {
        const int nc = min(a.pchunk, a.n_pairs - c0);
        // the B buffer is reused: every MMA of the previous chunk must be done
        finish_until(issued);
        const int base_q = issued;
        tc_fence_before();
        __syncthreads();
        for (int e = v; e < nc * (TC_B_PAIR_BYTES / 16); e += 128)
            cp_async_16(Bs + (size_t)e * 16, bmat + ((size_t)c0 * TC_B_PAIR_BYTES) + (size_t)e * 16);
        cp_async_commit();
        for (int j = v; j < nc; j += 128) {
            pt[j] = load_pair_tile(op, a.pairs[c0 + j], tile);
            sc[j] = inv_scale[c0 + j];
        }
        cp_async_wait_all();
        fence_proxy_async();
        __syncthreads();

        for (int j = 0; j < nc; ++j) {
            const int q = base_q + j;
            const int buf = q & 1;
            finish_until(q - 1);                       // pair q-2 used this A buffer and accumulator
            // A row of voxel v for pair q: z^k2, k2 = 0..15, split hi/lo
            const PVGeom G = pair_voxel(pt[j], o, op.ph);
            const float2 c = cis_turns_sfu(G.th0);
            const float2 an = make_float2(G.amp * c.x, G.amp * c.y);
            const float2 Zn = K1 > 1 ? cis_turns_sfu(G.dth2) : make_float2(1.f, 0.f);
            if (buf) { pa1 = an; pZ1 = Zn; pinv1 = sc[j]; }
            else { pa0 = an; pZ0 = Zn; pinv0 = sc[j]; }
            const float2 z = cis_turns(G.dth);
            unsigned char* Ab = As + buf * (2 * 2 * TC_KSTEP_BYTES_A);
            // powers z^0..z^15 as four chains stepped by z^4 (short dependency chains)
            const float2 z2 = cmul(z, z);
            const float2 z4 = cmul(z2, z2);
            float2 zp[4] = {make_float2(1.f, 0.f), z, z2, cmul(z2, z)};
#pragma unroll
            for (int grp = 0; grp < 4; ++grp) {       // powers 4 grp .. 4 grp + 3
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    split2<F16>(zp[u].x, zp[u].y, hi[u], lo[u]);
                    if (grp < 3) zp[u] = cmul(zp[u], z4);
                }
                const int s = grp / 2;                 // K step (k2 / 8)
                const uint32_t off = kmaj_off(v, (grp % 2) * 8);
                *reinterpret_cast<uint4*>(Ab + 0 * 2 * TC_KSTEP_BYTES_A + s * TC_KSTEP_BYTES_A + off) =
                    make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4*>(Ab + 1 * 2 * TC_KSTEP_BYTES_A + s * TC_KSTEP_BYTES_A + off) =
                    make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            const bool go = ok && issue;    // uniform
            if (go) ++committed;
            if (v == 0 && go) {
                tc_fence_after();
                const uint32_t d = tbase + (uint32_t)(buf * TC_N);
                const uint32_t a0 = smem_u32(Ab);
                const uint32_t b0 = smem_u32(Bs + (size_t)j * TC_B_PAIR_BYTES);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const uint64_t ahi = smem_desc(a0 + 0 * 2 * TC_KSTEP_BYTES_A + s * TC_KSTEP_BYTES_A);
                    const uint64_t alo = smem_desc(a0 + 1 * 2 * TC_KSTEP_BYTES_A + s * TC_KSTEP_BYTES_A);
                    const uint64_t bhi = smem_desc(b0 + 0 * 2 * TC_KSTEP_BYTES_B + s * TC_KSTEP_BYTES_B);
                    const uint64_t blo = smem_desc(b0 + 1 * 2 * TC_KSTEP_BYTES_B + s * TC_KSTEP_BYTES_B);
                    tc_mma(d, ahi, bhi, IDESC, s > 0 ? 1u : 0u);
                    tc_mma(d, ahi, blo, IDESC, 1u);
                    tc_mma(d, alo, bhi, IDESC, 1u);
                }
                tc_commit(&bar[buf]);
            }
        }
        issued = base_q + nc;
    }
    finish_until(issued);
    pdl_launch_dependents();

    if (!ok && v == 0) atomicOr(op.err, ERRF_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 32);
    }

    const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
    if (!ok || ix >= op.g.nx || iy >= op.g.ny || iz >= op.g.nz) return;
    const size_t n = ((size_t)iz * op.g.ny + iy) * op.g.nx + ix;
    if (a.s) {
        const float2 sv = a.s[n];
        const float zr = fmaf(-a.step, g.x, sv.x), zi = fmaf(-a.step, g.y, sv.y);
        const float mag = sqrtf(zr * zr + zi * zi);
        float2 out = make_float2(0.f, 0.f);
        if (mag > a.alpha) {
            const float f = (1.0f - a.alpha / mag) * a.shrink;
            out = make_float2(zr * f, zi * f);
        }
        a.s[n] = out;
    } else {
        a.g_out[n] = g;
    }
}

size_t adj_tc_smem_bytes(int pchunk)
{
    return (size_t)2 * 2 * 2 * TC_KSTEP_BYTES_A + (size_t)pchunk * TC_B_PAIR_BYTES + (size_t)pchunk * sizeof(PairTile) +
           (size_t)((pchunk + 1) & ~1) * sizeof(float) + 2 * sizeof(uint64_t) + 16;
}

size_t adj_tc_bmat_bytes(int n_pairs) { return (size_t)n_pairs * TC_B_PAIR_BYTES; }

template <int K1, bool F16>
static const void* adj_tc_ptr1() { return (const void*)adj_tc_kernel<K1, F16>; }

const void* adj_tc_kernel_ptr(int K1, bool f16)
{
    switch (K1) {
    case 1: return f16 ? adj_tc_ptr1<1, true>() : adj_tc_ptr1<1, false>();
    case 2: return f16 ? adj_tc_ptr1<2, true>() : adj_tc_ptr1<2, false>();
    case 3: return f16 ? adj_tc_ptr1<3, true>() : adj_tc_ptr1<3, false>();
    case 4: return f16 ? adj_tc_ptr1<4, true>() : adj_tc_ptr1<4, false>();
    case 5: return f16 ? adj_tc_ptr1<5, true>() : adj_tc_ptr1<5, false>();
    case 6: return f16 ? adj_tc_ptr1<6, true>() : adj_tc_ptr1<6, false>();
    case 7: return f16 ? adj_tc_ptr1<7, true>() : adj_tc_ptr1<7, false>();
    case 8: return f16 ? adj_tc_ptr1<8, true>() : adj_tc_ptr1<8, false>();
    default: return nullptr;
    }
}

cudaError_t launch_adjoint_tc(const OpDesc& op, const AdjArgs& a, bool f16, const float2* r, unsigned char* bmat,
                              float* inv_scale, size_t smem, cudaStream_t st)
{
    const void* prep = f16 ? (const void*)adj_tc_prep_kernel<true> : (const void*)adj_tc_prep_kernel<false>;
    int np = a.n_pairs;
    void* pargs[] = {(void*)&op, (void*)&r, (void*)&np, (void*)&bmat, (void*)&inv_scale};
    cudaError_t e = launch_pdl(prep, dim3(a.n_pairs), dim3(128), 0, st, pargs);
    if (e != cudaSuccess) return e;
    const void* fn = adj_tc_kernel_ptr(op.K1, f16);
    if (!fn) return cudaErrorInvalidValue;
    const unsigned char* bm = bmat;
    const float* is = inv_scale;
    void* args[] = {(void*)&op, (void*)&a, (void*)&bm, (void*)&is};
    return launch_pdl(fn, dim3(op.g.n_tiles), dim3(128), smem, st, args);
}

}  // namespace nfm
