// Forward and adjoint for an arbitrary list of frequencies f_k (Eq. 2 with no
// assumption on the spacing; p(f_k) any complex spectrum).  Without a common
// frequency step there is no phasor recurrence: every element gets its own
// phase
//
//     theta_k = frac( B_k + f_k delta / c ),   B_k = frac(f_k |v_T|/c) + frac(f_k |v_R|/c)
//
// with the tile-relative distance offset delta of the uniform path and the
// per-(antenna, tile, frequency) reduced phases taken from an FP64 table.  The
// product f_k delta / c is split so that only one FP32 rounding at magnitude
// <= 1 turn remains; the phasor comes from the SFU sine/cosine (absolute error
// ~4e-7; it starts no recurrence, so the error is not amplified).
#include "nfm_kernels.cuh"

namespace nfm {

// frac(f_k d / c) for every (antenna, tile, k), FP64 then rounded to FP32.
__global__ void antk_setup_kernel(GridDesc g, AntSetup a, const double* fk_over_c, int K, float* out)
{
    const long long total = (long long)a.n_ant * g.n_tiles * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        const long long at = i / K;
        const int tile = (int)(at % g.n_tiles);
        const int ant = (int)(at / g.n_tiles);
        int tx, ty, tz;
        tile_coords(g, tile, tx, ty, tz);
        const double cx = a.x0 + (tx * TILE_X + 0.5 * (TILE_X - 1)) * a.dx;
        const double cy = a.y0 + (ty * TILE_Y + 0.5 * (TILE_Y - 1)) * a.dy;
        const double cz = a.z0 + (tz * TILE_Z + 0.5 * (TILE_Z - 1)) * a.dz;
        const double vx = a.ant_xyz[3 * ant] - cx, vy = a.ant_xyz[3 * ant + 1] - cy, vz = a.ant_xyz[3 * ant + 2] - cz;
        double b = fk_over_c[k] * sqrt(vx * vx + vy * vy + vz * vz);
        b -= rint(b);
        out[i] = (float)b;
    }
}

cudaError_t launch_antk_setup(const GridDesc& g, const AntSetup& a, const double* fk_over_c, int K, float* out,
                              cudaStream_t st)
{
    long long total = (long long)a.n_ant * g.n_tiles * K;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    antk_setup_kernel<<<blocks, 256, 0, st>>>(g, a, fk_over_c, K, out);
    return cudaGetLastError();
}

// theta = frac(Bk + fkc * delta) with fkc = f_k/c as hi + lo
__device__ __forceinline__ float gen_phase(float Bk, float2 fkc, float delta)
{
    const float p = __fmul_rn(fkc.x, delta);    // rounded product: its error pe is added back below
    const float pe = fmaf(fkc.x, delta, -p);
    return frac_turns((Bk + (p - rintf(p))) + fmaf(fkc.y, delta, pe));
}

// Pair constants needed here: geometry from PairTile, phases from the table.
__device__ __forceinline__ float pair_delta_amp(const PairTile& P, const VoxelOffset& o, float& amp)
{
    float rsT, rsR;
    const float dT = antenna_delta(P.vTx, P.vTy, P.vTz, P.dcT, P.dcT2, o, rsT);
    const float dR = antenna_delta(P.vRx, P.vRy, P.vRz, P.dcR, P.dcR2, o, rsR);
    amp = INV_4PI * rsT * rsR;
    return dT + dR;
}

__device__ __forceinline__ void pair_table_rows(const OpDesc& op, const GenDesc& gd, int pair, int tile,
                                                const float*& bt, const float*& br)
{
    if (pair < 0 || pair >= op.P) {
        atomicOr(op.err, ERRF_PAIR);
        pair = 0;
    }
    const int t = pair / op.R, r = pair - (pair / op.R) * op.R;
    bt = gd.antk + ((size_t)t * op.g.n_tiles + tile) * op.K;
    br = gd.antk + ((size_t)(op.T + r) * op.g.n_tiles + tile) * op.K;
}

// Forward: grid (pair groups of 8, voxel-tile chunks), 256 threads; warp p =
// pair p of the group, lane owns frequencies lane, lane + 32, ... (K <= 128).
__global__ void __launch_bounds__(256) fwd_general_kernel(OpDesc op, GenDesc gd, FwdArgs a)
{
    constexpr int PC = FWD_PC;
    __shared__ float2 u_s[TILE_V][PC];     // amp * s
    __shared__ float d_s[TILE_V][PC];      // delta
    __shared__ float Bk_s[PC][GEN_MAX_K];
    __shared__ float2 fkc_s[GEN_MAX_K];
    __shared__ PairTile pt_s[PC];
    __shared__ int pair_s[PC];
    const int tid = threadIdx.x, p = tid / 32, lane = tid % 32;
    const int group = blockIdx.x, chunk = blockIdx.y;
    const int t_begin = chunk * a.tiles_base + min(chunk, a.tiles_rem);
    const int t_end = t_begin + a.tiles_base + (chunk < a.tiles_rem ? 1 : 0);
    for (int k = tid; k < op.K; k += 256) fkc_s[k] = gd.fkc[k];
    pdl_wait();
    if (tid < PC) {
        const int slot = group * PC + tid;
        pair_s[tid] = slot < a.n_pairs ? a.pairs[slot] : -1;
    }
    float2 acc[GEN_MAX_K / 32];
#pragma unroll
    for (int j = 0; j < GEN_MAX_K / 32; ++j) acc[j] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int tile = t_begin; tile < t_end; ++tile) {
        int tx, ty, tz;
        tile_coords(op.g, tile, tx, ty, tz);
        if (tid < PC) {
            const int pair = pair_s[tid];
            pt_s[tid] = load_pair_tile(op, pair < 0 ? 0 : pair, tile);
        }
        for (int e = tid; e < PC * op.K; e += 256) {
            const int i = e / op.K, k = e - (e / op.K) * op.K;
            const int pair = pair_s[i];
            const float *bt, *br;
            pair_table_rows(op, gd, pair < 0 ? 0 : pair, tile, bt, br);
            Bk_s[i][k] = frac_turns(bt[k] + br[k]);
        }
        __syncthreads();
        for (int e = tid; e < TILE_V * PC; e += 256) {
            const int i = e % PC, v = e / PC;
            const int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y);
            const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
            float2 sv = make_float2(0.f, 0.f);
            if (pair_s[i] >= 0 && ix < op.g.nx && iy < op.g.ny && iz < op.g.nz)
                sv = a.s[((size_t)iz * op.g.ny + iy) * op.g.nx + ix];
            float amp;
            const float dl = pair_delta_amp(pt_s[i], voxel_offset(op.g, lx, ly, lz), amp);
            u_s[v][i] = make_float2(amp * sv.x, amp * sv.y);
            d_s[v][i] = dl;
        }
        __syncthreads();
        for (int v = 0; v < TILE_V; ++v) {
            const float2 u = u_s[v][p];
            const float dl = d_s[v][p];
#pragma unroll
            for (int j = 0; j < GEN_MAX_K / 32; ++j) {
                const int k = lane + 32 * j;
                if (k < op.K) {
                    const float2 c = cis_turns_sfu(gen_phase(Bk_s[p][k], fkc_s[k], dl));
                    const float2 t = cmul_conj(u, c);      // u e^{-j 2 pi theta}
                    acc[j].x += t.x;
                    acc[j].y += t.y;
                }
            }
        }
        __syncthreads();
    }
    pdl_launch_dependents();
    const int slot = group * PC + p;
    if (slot < a.n_pairs) {
#pragma unroll
        for (int j = 0; j < GEN_MAX_K / 32; ++j) {
            const int k = lane + 32 * j;
            if (k < op.K) a.partial[((size_t)chunk * a.n_slots + slot) * op.K + k] = acc[j];
        }
    }
}

// Adjoint: one CTA = one tile, 128 threads = 128 voxels; pairs staged in chunks.
__global__ void __launch_bounds__(128) adj_general_kernel(OpDesc op, GenDesc gd, AdjArgs a)
{
    constexpr int PCH = GEN_ADJ_PCHUNK;
    __shared__ float2 r_s[PCH][GEN_MAX_K];
    __shared__ float Bk_s[PCH][GEN_MAX_K];
    __shared__ float2 fkc_s[GEN_MAX_K];
    __shared__ PairTile pt_s[PCH];
    const int tile = blockIdx.x;
    int tx, ty, tz;
    tile_coords(op.g, tile, tx, ty, tz);
    const int v = threadIdx.x;
    const int lx = v % TILE_X, ly = (v / TILE_X) % TILE_Y, lz = v / (TILE_X * TILE_Y);
    const VoxelOffset o = voxel_offset(op.g, lx, ly, lz);
    for (int k = v; k < op.K; k += 128) fkc_s[k] = gd.fkc[k];
    pdl_wait();
    float2 g = make_float2(0.f, 0.f);
    for (int c0 = 0; c0 < a.n_pairs; c0 += PCH) {
        const int nc = min(PCH, a.n_pairs - c0);
        __syncthreads();
        for (int e = v; e < nc * op.K; e += 128) {
            const int j = e / op.K, k = e - (e / op.K) * op.K;
            float2 rv = a.r[(size_t)(c0 + j) * op.K + k];
            if (op.pulse) rv = cmul_conj(rv, op.pulse[k]);   // conj(p_k) r
            r_s[j][k] = rv;
            const float *bt, *br;
            pair_table_rows(op, gd, a.pairs[c0 + j], tile, bt, br);
            Bk_s[j][k] = frac_turns(bt[k] + br[k]);
        }
        for (int j = v; j < nc; j += 128) pt_s[j] = load_pair_tile(op, a.pairs[c0 + j], tile);
        __syncthreads();
        for (int j = 0; j < nc; ++j) {
            float amp;
            const float dl = pair_delta_amp(pt_s[j], o, amp);
            float2 h0 = make_float2(0.f, 0.f), h1 = h0;
            int k = 0;
            for (; k + 1 < op.K; k += 2) {         // two independent sums for ILP
                const float2 c0v = cis_turns_sfu(gen_phase(Bk_s[j][k], fkc_s[k], dl));
                const float2 c1v = cis_turns_sfu(gen_phase(Bk_s[j][k + 1], fkc_s[k + 1], dl));
                const float2 t0 = cmul(c0v, r_s[j][k]), t1 = cmul(c1v, r_s[j][k + 1]);
                h0.x += t0.x; h0.y += t0.y;
                h1.x += t1.x; h1.y += t1.y;
            }
            if (k < op.K) {
                const float2 t0 = cmul(cis_turns_sfu(gen_phase(Bk_s[j][k], fkc_s[k], dl)), r_s[j][k]);
                h0.x += t0.x; h0.y += t0.y;
            }
            g.x = fmaf(amp, h0.x + h1.x, g.x);
            g.y = fmaf(amp, h0.y + h1.y, g.y);
        }
    }
    pdl_launch_dependents();
    const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
    if (ix >= op.g.nx || iy >= op.g.ny || iz >= op.g.nz) return;
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

cudaError_t launch_fwd_general(const OpDesc& op, const GenDesc& gd, const FwdArgs& a, dim3 grid, cudaStream_t st)
{
    void* args[] = {(void*)&op, (void*)&gd, (void*)&a};
    return launch_pdl((const void*)fwd_general_kernel, grid, dim3(256), 0, st, args);
}

cudaError_t launch_adj_general(const OpDesc& op, const GenDesc& gd, const AdjArgs& a, cudaStream_t st)
{
    void* args[] = {(void*)&op, (void*)&gd, (void*)&a};
    return launch_pdl((const void*)adj_general_kernel, dim3(op.g.n_tiles), dim3(128), 0, st, args);
}

const void* fwd_general_ptr() { return (const void*)fwd_general_kernel; }

}  // namespace nfm
