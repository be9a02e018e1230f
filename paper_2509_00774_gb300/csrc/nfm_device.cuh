// Device-side building blocks of the matrix-free observation operator (Eq. 2).
//
// A[m][n] = p(f_k) exp(-j 2 pi f_k (dT + dR)/c) / (4 pi dT dR),  m = (pair, k)
//
// Precision scheme (FP32 arithmetic in every per-element loop):
//  * Voxels are grouped in tiles of TILE_X x TILE_Y x TILE_Z.  For each
//    (antenna, tile) a FP64 set-up kernel stores v = r_a - r_c (r_c = tile
//    centre), |v| and the reduced phases f0|v|/c, df|v|/c, K2 df|v|/c.
//  * Per voxel, d = |r_a - r_n| is written as d = |v| + delta with
//    delta = q / (|v| + d), q = |u|^2 - 2 v.u, u = r_n - r_c.  delta is a few
//    centimetres, so its FP32 rounding is ~1e-9 m although d itself is ~0.5 m.
//  * The phase in cycles is f_k (D_c + delta)/c with D_c = |v_T| + |v_R|; the
//    D_c part comes from the FP64 tables and is reduced mod 1 before FP32.
//  * Frequencies are equally spaced, f_k = f0 + k df.  With k = k1 K2 + k2 the
//    phasor exp(-j 2 pi f_k D/c) is built from a base value, a block step
//    W = exp(-j 2 pi K2 df D/c) and a fine step w = exp(-j 2 pi df D/c), each
//    from its own reduced phase, so no recurrence runs more than K2 steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nfm {

constexpr int K2 = 16;                                 // frequencies per block
constexpr int MAX_K1 = 8;                              // K <= 128
constexpr int TILE_X = 8, TILE_Y = 4, TILE_Z = 4;      // geometry tile (voxels)
constexpr int TILE_V = TILE_X * TILE_Y * TILE_Z;       // 128
constexpr float INV_4PI = 0.0795774715459476679f;      // 1/(4 pi)

// Per (antenna, tile) constants written by the FP64 set-up kernel.
struct __align__(16) AntTile {
    float vx, vy, vz;      // r_a - r_c (metres)
    float dc;              // |r_a - r_c|
    float dc2;             // |r_a - r_c|^2
    float b;               // frac(f0 dc / c)                 (cycles, in [-1/2, 1/2])
    float s_hi, s_lo;      // frac(df dc / c) as hi + lo
    float s2_hi, s2_lo;    // frac(K2 df dc / c) as hi + lo
    float pad0, pad1;
};

// The leading 32 bytes of an AntTile: what the expansion operator reads (no K2 step).
struct __align__(16) AntHead {
    float vx, vy, vz, dc;
    float dc2, b, s_hi, s_lo;
};
static_assert(sizeof(AntHead) == 32, "AntHead is the first two 16-byte words of an AntTile");

// Per (pair, tile) constants: the TX and RX AntTile folded together.
struct __align__(16) PairTile {
    float vTx, vTy, vTz, dcT, dcT2;
    float vRx, vRy, vRz, dcR, dcR2;
    float B;               // frac(f0 D_c / c)
    float S_hi, S_lo;      // frac(df D_c / c)
    float S2_hi, S2_lo;    // frac(K2 df D_c / c)
    float pad;
};

struct GridDesc {
    int nx, ny, nz;
    int tiles_x, tiles_y, tiles_z;
    int n_tiles;
    float dx_hi, dx_lo, dy_hi, dy_lo, dz_hi, dz_lo;
    // n / tiles_x = umulhi(n, mx) and n / tiles_y = umulhi(n, my) for 0 <= n < n_tiles (division by an
    // invariant integer with a rounded-up reciprocal: exact while n * divisor < 2^32); 0 = divide
    unsigned mx, my;
    // Explicit voxel positions: voxel n sits in slot n % 128 of tile n / 128 (tiles_x = n_tiles, nx = N,
    // ny = nz = 1) and pts[n] (padded to whole tiles) holds its offset from the tile centre as
    // (ux, uy, uz, |u|^2) in FP32; nullptr for a regular grid.
    const float4* pts = nullptr;
};

struct PhaseConsts {
    float f0c_hi, f0c_lo;  // f0 / c  (cycles per metre) as hi + lo
    float dfc;             // df / c
    float dfc2;            // K2 df / c
};

// Operator description passed by value to every kernel.
struct OpDesc {
    GridDesc g;
    PhaseConsts ph;
    const AntTile* ant;    // [(T + R) * n_tiles]: TX rows first, then RX rows
    const float2* pulse;   // [K] or nullptr (p = 1)
    int T, R, K, K1, P;
    int* err;              // device error flags
    unsigned long long wait_ns = 1000000000ull;   // limit of one bounded wait on the tensor core
    int hooks = 0;         // test hooks (HOOK_*), 0 in normal operation
    long long n_vox = 0;   // N: extent of s and g (checked in the bounds-checked build)
    long long m_rows = 0;  // P K: extent of the full measurement vector (checked in the bounds-checked build)
};

enum : int { ERRF_PAIR = 1, ERRF_TIMEOUT = 2, ERRF_BOUNDS = 4 };
// HOOK_TC_SKIP_ISSUE: the tensor-core kernels issue no MMA and no commit, so their bounded waits run
// out and the timeout path runs (no outstanding tensor-core work, nothing faults or hangs)
enum : int { HOOK_TC_SKIP_ISSUE = 1, HOOK_SHRINK_EXTENTS = 2 };

// Bounds-checked build (-DNFM_BOUNDS_CHECK): a checked global index is compared with the extent the host
// passed for that buffer; an index outside it raises ERRF_BOUNDS and is replaced by 0, an element that
// exists, so the access stays inside the buffer.  In the normal build the check compiles away.
#ifdef NFM_BOUNDS_CHECK
__device__ __forceinline__ long long nfm_checked(long long i, long long n, int* err)
{
    if (i < 0 || i >= n) {
        atomicOr(err, ERRF_BOUNDS);
        return 0;
    }
    return i;
}
#define NFM_IDX(i, n, err) nfm_checked((long long)(i), (long long)(n), (err))
#else
#define NFM_IDX(i, n, err) (i)
#endif

__device__ __forceinline__ float frac_turns(float x) { return x - rintf(x); }

// (cos 2 pi t, sin 2 pi t) for t in turns, |t| <= 1.
// Method: reduce to the nearest quarter turn q/4 (exact: Sterbenz), evaluate
// the Taylor series of sin and cos about 0 on x = 2 pi (t - q/4) in
// [-pi/4, pi/4] (sin to x^9, cos to x^8; truncation < 3e-8), then rotate by
// q quarter turns.
__device__ __forceinline__ float2 cis_turns(float t)
{
    float q = rintf(4.0f * t);
    float r = fmaf(-0.25f, q, t);
    float x = r * 6.28318530717958648f;
    float x2 = x * x;
    float ps = fmaf(x2, 2.75573192e-6f, -1.98412698e-4f);   //  1/9!, -1/7!
    ps = fmaf(x2, ps, 8.33333333e-3f);                       //  1/5!
    ps = fmaf(x2, ps, -1.66666667e-1f);                      // -1/3!
    float sn = fmaf(x * x2, ps, x);
    float pc = fmaf(x2, 2.48015873e-5f, -1.38888889e-3f);   //  1/8!, -1/6!
    pc = fmaf(x2, pc, 4.16666667e-2f);                       //  1/4!
    pc = fmaf(x2, pc, -0.5f);                                // -1/2!
    float cs = fmaf(x2, pc, 1.0f);
    int iq = __float2int_rn(q) & 3;
    float c = (iq & 1) ? sn : cs;
    float s = (iq & 1) ? cs : sn;
    // rotation by iq quarter turns: 0:(c,s) 1:(-s,c) 2:(-c,-s) 3:(s,-c)
    float co = (iq == 1 || iq == 2) ? -c : c;
    float si = (iq >= 2) ? -s : s;
    return make_float2(co, si);
}

// (cos 2 pi t, sin 2 pi t) for |t| <= 1/2 from the SFU sine/cosine
// approximations (absolute error about 4e-7 on [-pi, pi]).  Used only where the
// phasor starts a sequence and its error is not amplified by a recurrence.
__device__ __forceinline__ float2 cis_turns_sfu(float t)
{
    float s, c;
    __sincosf(6.28318530717958648f * t, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// a * conj(b)
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// Error-free sum a + b = s + e (Knuth TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ PairTile fold_pair_tile(const AntTile& t, const AntTile& r)
{
    PairTile p;
    p.pad = 0.f;
    p.vTx = t.vx; p.vTy = t.vy; p.vTz = t.vz; p.dcT = t.dc; p.dcT2 = t.dc2;
    p.vRx = r.vx; p.vRy = r.vy; p.vRz = r.vz; p.dcR = r.dc; p.dcR2 = r.dc2;
    p.B = frac_turns(t.b + r.b);
    float h, e;
    two_sum(t.s_hi, r.s_hi, h, e);
    p.S_hi = frac_turns(h);
    p.S_lo = e + (t.s_lo + r.s_lo);
    two_sum(t.s2_hi, r.s2_hi, h, e);
    p.S2_hi = frac_turns(h);
    p.S2_lo = e + (t.s2_lo + r.s2_lo);
    return p;
}

// The same from the leading words only (S2 left zero; the expansion operator does not use it).
__device__ __forceinline__ PairTile fold_pair_head(const AntHead& t, const AntHead& r)
{
    PairTile p;
    p.pad = 0.f;
    p.vTx = t.vx; p.vTy = t.vy; p.vTz = t.vz; p.dcT = t.dc; p.dcT2 = t.dc2;
    p.vRx = r.vx; p.vRy = r.vy; p.vRz = r.vz; p.dcR = r.dc; p.dcR2 = r.dc2;
    p.B = frac_turns(t.b + r.b);
    float h, e;
    two_sum(t.s_hi, r.s_hi, h, e);
    p.S_hi = frac_turns(h);
    p.S_lo = e + (t.s_lo + r.s_lo);
    p.S2_hi = 0.f;
    p.S2_lo = 0.f;
    return p;
}

// Position of a voxel relative to its tile centre, from its local index.
struct __align__(16) VoxelOffset {
    float ux, uy, uz, uu;
};

// (tz: the z extent of the block the offset is taken in; TILE_Z for the tiles)
__device__ __forceinline__ VoxelOffset voxel_offset(const GridDesc& g, int lx, int ly, int lz, int tz = TILE_Z)
{
    float ox = (float)lx - 0.5f * (TILE_X - 1);
    float oy = (float)ly - 0.5f * (TILE_Y - 1);
    float oz = (float)lz - 0.5f * (float)(tz - 1);
    VoxelOffset o;
    o.ux = fmaf(ox, g.dx_hi, ox * g.dx_lo);
    o.uy = fmaf(oy, g.dy_hi, oy * g.dy_lo);
    o.uz = fmaf(oz, g.dz_hi, oz * g.dz_lo);
    o.uu = fmaf(o.ux, o.ux, fmaf(o.uy, o.uy, o.uz * o.uz));
    return o;
}

// Per (pair, voxel): amplitude 1/(4 pi dT dR) and the three reduced phases.
struct PVGeom {
    float amp;
    float th0;   // f0 D / c          (turns, reduced)
    float dth;   // df D / c          (turns, reduced)
    float dth2;  // K2 df D / c       (turns, reduced)
};

// d - dc and 1/d from q = d^2 - dc^2 (no cancellation: d - dc = q / (dc + d))
__device__ __forceinline__ float antenna_delta_q(float q, float dc, float dc2, float& rs)
{
    float d2 = dc2 + q;
    rs = rsqrtf(d2);                           // 1/d
    float d = d2 * rs;
    return __fdividef(q, dc + d);              // d - dc
}

__device__ __forceinline__ float antenna_delta(float vx, float vy, float vz, float dc, float dc2,
                                               const VoxelOffset& o, float& rs)
{
    float vu = fmaf(vx, o.ux, fmaf(vy, o.uy, vz * o.uz));
    float q = fmaf(-2.0f, vu, o.uu);           // d^2 - dc^2 = |u|^2 - 2 v.u
    return antenna_delta_q(q, dc, dc2, rs);
}

__device__ __forceinline__ PVGeom pair_voxel(const PairTile& pt, const VoxelOffset& o, const PhaseConsts& ph)
{
    float rsT, rsR;
    float dT = antenna_delta(pt.vTx, pt.vTy, pt.vTz, pt.dcT, pt.dcT2, o, rsT);
    float dR = antenna_delta(pt.vRx, pt.vRy, pt.vRz, pt.dcR, pt.dcR2, o, rsR);
    float delta = dT + dR;
    PVGeom gv;
    gv.amp = INV_4PI * rsT * rsR;
    // f0 (D_c + delta)/c: exact product split so only one rounding at |x| <= 1
    float p = __fmul_rn(ph.f0c_hi, delta);      // rounded product: its error pe is added back below
    float pe = fmaf(ph.f0c_hi, delta, -p);
    float th = (pt.B + (p - rintf(p))) + fmaf(ph.f0c_lo, delta, pe);
    gv.th0 = frac_turns(th);
    gv.dth = frac_turns(pt.S_hi + fmaf(ph.dfc, delta, pt.S_lo));
    gv.dth2 = frac_turns(pt.S2_hi + fmaf(ph.dfc2, delta, pt.S2_lo));
    return gv;
}

__device__ __forceinline__ void tile_coords(const GridDesc& g, int tile, int& tx, int& ty, int& tz)
{
    const int rest = g.mx ? (int)__umulhi((unsigned)tile, g.mx) : tile / g.tiles_x;
    tx = tile - rest * g.tiles_x;
    tz = g.my ? (int)__umulhi((unsigned)rest, g.my) : rest / g.tiles_y;
    ty = rest - tz * g.tiles_y;
}

// Programmatic dependent launch: wait until the preceding kernel in the stream
// has completed and its writes are visible (no-op without the launch attribute),
// and let the next kernel begin launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asynchronous global -> shared copies (completion tracked per thread).
__device__ __forceinline__ void cp_async_8(void* smem_dst, const void* gmem_src, bool valid)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    int n = valid ? 8 : 0;   // 0 source bytes: the destination is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem_src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gmem_src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
// The same through L1 (.ca), for data that many CTAs of an SM read (the minibatch residual).
__device__ __forceinline__ void cp_async_16_ca(void* smem_dst, const void* gmem_src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Row of the AntTile table for (pair, tile): TX row and RX row.  An
// out-of-range pair raises the flag and falls back to pair 0.
__device__ __forceinline__ void pair_rows(const OpDesc& op, int pair, int tile, const AntTile*& at, const AntTile*& ar)
{
    if (pair < 0 || pair >= op.P) {
        atomicOr(op.err, ERRF_PAIR);
        pair = 0;
    }
    int t = pair / op.R;
    int r = pair - t * op.R;
    at = op.ant + (size_t)t * op.g.n_tiles + tile;
    ar = op.ant + (size_t)(op.T + r) * op.g.n_tiles + tile;
}

// Load the (pair, tile) constants; an out-of-range pair raises the flag and
// falls back to pair 0 so every access stays in bounds.
__device__ __forceinline__ PairTile load_pair_tile(const OpDesc& op, int pair, int tile)
{
    if (pair < 0 || pair >= op.P) {
        atomicOr(op.err, ERRF_PAIR);
        pair = 0;
    }
    int t = pair / op.R;
    int r = pair - t * op.R;
    AntTile at = op.ant[(size_t)t * op.g.n_tiles + tile];
    AntTile ar = op.ant[(size_t)(op.T + r) * op.g.n_tiles + tile];
    return fold_pair_tile(at, ar);
}

}  // namespace nfm
