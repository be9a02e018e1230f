// Per-(pair, voxel) geometry of the Chebyshev-expansion operator and the
// tile phasor P_k = exp(-j 2 pi k df D_c / c) (shared by the CUDA-core and the
// tensor-core kernels of the expansion).
#pragma once
#include "nfm_device.cuh"

namespace nfm {

// amplitude, reduced base phase (f_0 D_c + f_c delta)/c (turns) and delta = D - D_c of one (pair, voxel).
// With f_k = f_0 + k df and the band centre f_c = f_0 + k_c df,
//   f_k D = f_0 D_c + f_c delta + k df D_c + (k - k_c) df delta,
// so the phase left to the expansion, (k - k_c) df delta / c, is centred on zero over the band.
struct ChebVoxel {
    float amp, th0, delta;
};

// ... from d - d_c (dT, dR) and 1/d (rsT, rsR) of the TX and the RX antenna
__device__ __forceinline__ ChebVoxel cheb_voxel_d(const PairTile& pt, float dT, float rsT, float dR, float rsR,
                                                  float fc_hi, float fc_lo)
{
    ChebVoxel c;
    c.delta = dT + dR;
    c.amp = INV_4PI * rsT * rsR;
    // B = f_0 D_c / c (reduced) plus f_c delta / c: the fused fc_hi delta - n, n the integer nearest the
    // product, rounds once at |x| <= 1/2 (f_c / c = fc_hi + fc_lo)
    const float n = rintf(fc_hi * c.delta);
    const float th = fmaf(fc_lo, c.delta, pt.B + fmaf(fc_hi, c.delta, -n));
    c.th0 = frac_turns(th);
    return c;
}

// ... from the voxel's q = d^2 - d_c^2 to the TX (qT) and the RX (qR) antenna
__device__ __forceinline__ ChebVoxel cheb_voxel_q(const PairTile& pt, float qT, float qR, float fc_hi, float fc_lo)
{
    float rsT, rsR;
    const float dT = antenna_delta_q(qT, pt.dcT, pt.dcT2, rsT);
    const float dR = antenna_delta_q(qR, pt.dcR, pt.dcR2, rsR);
    return cheb_voxel_d(pt, dT, rsT, dR, rsR, fc_hi, fc_lo);
}

// ... from the voxel's offset u to the tile centre: q = |u|^2 - 2 v.u, v = r_a - r_c (one antenna after
// the other: the tensor-core forward measured 10% slower with both q formed first)
__device__ __forceinline__ ChebVoxel cheb_voxel(const PairTile& pt, const VoxelOffset& o, float fc_hi, float fc_lo)
{
    float rsT, rsR;
    const float dT = antenna_delta(pt.vTx, pt.vTy, pt.vTz, pt.dcT, pt.dcT2, o, rsT);
    const float dR = antenna_delta(pt.vRx, pt.vRy, pt.vRz, pt.dcR, pt.dcR2, o, rsR);
    return cheb_voxel_d(pt, dT, rsT, dR, rsR, fc_hi, fc_lo);
}

// The base phase advanced by k_c steps, B + k_c S (k_c = (K - 1)/2, the band centre), so that the tile
// phasors can run from the band centre: P_k = e^{-j 2 pi k_c S} e^{-j 2 pi (k - k_c) S}, the first factor
// carried by every voxel's base phase, the second conjugate between k and its mirror K-1-k.
__device__ __forceinline__ void centre_base_phase(PairTile& p, int K)
{
    const float kc = 0.5f * (float)(K - 1);
    const float q = __fmul_rn(kc, p.S_hi);      // rounded product: its error e is added back below
    const float e = fmaf(kc, p.S_hi, -q);
    p.B = frac_turns((p.B + (q - rintf(q))) + fmaf(kc, p.S_lo, e));
}

// The pair tile as the adjoint uses it: antenna vectors scaled by -2 (exact), for cheb_voxel_m2 below, and
// the base phase centred on the band.
__device__ __forceinline__ PairTile pair_tile_adj(PairTile p, int K)
{
    p.vTx *= -2.f; p.vTy *= -2.f; p.vTz *= -2.f;
    p.vRx *= -2.f; p.vRy *= -2.f; p.vRz *= -2.f;
    centre_base_phase(p, K);
    return p;
}

// cheb_voxel of a pair tile from pair_tile_adj: q = |u|^2 + (-2 v).u in three FMAs per antenna
__device__ __forceinline__ ChebVoxel cheb_voxel_m2(const PairTile& pm, const VoxelOffset& o, float fc_hi, float fc_lo)
{
    const float qT = fmaf(pm.vTx, o.ux, fmaf(pm.vTy, o.uy, fmaf(pm.vTz, o.uz, o.uu)));
    const float qR = fmaf(pm.vRx, o.ux, fmaf(pm.vRy, o.uy, fmaf(pm.vRz, o.uz, o.uu)));
    return cheb_voxel_q(pm, qT, qR, fc_hi, fc_lo);
}

// (cos, sin)(2 pi k df D_c / c) from the reduced step phase S = S_hi + S_lo of the
// pair tile: k S_hi split exactly (FMA remainder), so one rounding at |x| <= 1/2.
// (kf: an integer or half-integer step count)
__device__ __forceinline__ float2 tile_step_cis_f(const PairTile& pt, float kf)
{
    const float p = __fmul_rn(kf, pt.S_hi);     // rounded product: its error e is added back below
    const float e = fmaf(kf, pt.S_hi, -p);
    const float ph = (p - rintf(p)) + fmaf(kf, pt.S_lo, e);
    return cis_turns_sfu(ph);
}

__device__ __forceinline__ float2 tile_step_cis(const PairTile& pt, int k) { return tile_step_cis_f(pt, (float)k); }

// The same phasor from the Taylor-series cis_turns (error ~1e-7), for a step that a recurrence repeats.
__device__ __forceinline__ float2 tile_step_cis_exact(const PairTile& pt, int k)
{
    const float kf = (float)k;
    const float p = __fmul_rn(kf, pt.S_hi);     // rounded product: its error e is added back below
    const float e = fmaf(kf, pt.S_hi, -p);
    const float ph = (p - rintf(p)) + fmaf(kf, pt.S_lo, e);
    return cis_turns(ph);
}

// Gradient step and prox of one voxel's iterate (Eq. 5 with the regulariser extended as Sec. III
// allows): z = s - step g, the soft threshold at alpha (l1 term), the group shrink at alpha_g over the
// 2 x 2 x 1 voxel block held by lanes lane, lane ^ 1, lane ^ 8, lane ^ 9 of the warp (thread = voxel
// v of an 8 x 4 x 4 tile with lx = v % 8, ly = (v / 8) % 4; tile origins are even, so blocks never
// straddle tiles), then the elastic-net scaling.  With alpha_g > 0 every lane of the warp must call
// it; voxels outside the grid pass in = false and add nothing to their block's norm.
__device__ __forceinline__ float2 step_prox(float2 s, float gr, float gi, float step, float alpha, float alpha_g,
                                            float shrink, bool in)
{
    const float zr = fmaf(-step, gr, s.x), zi = fmaf(-step, gi, s.y);
    const float mag = sqrtf(zr * zr + zi * zi);
    float f = mag > alpha ? 1.0f - alpha / mag : 0.f;
    if (alpha_g > 0.f) {
        const float u2 = in ? f * f * (zr * zr + zi * zi) : 0.f;
        float n2 = u2 + __shfl_xor_sync(0xffffffffu, u2, 1);
        n2 += __shfl_xor_sync(0xffffffffu, n2, 8);
        const float gn = sqrtf(n2);
        f *= gn > alpha_g ? 1.0f - alpha_g / gn : 0.f;
    }
    const float sc = f * shrink;
    return make_float2(zr * sc, zi * sc);
}

}  // namespace nfm
