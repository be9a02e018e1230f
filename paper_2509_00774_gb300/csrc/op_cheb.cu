// Matrix-free A_B s and A_B^H r (Eq. 2) by a tile-local Chebyshev expansion of
// the frequency dependence (equally spaced frequencies f_k = f0 + k df).
//
// For a (pair, tile) with centre path length D_c and a voxel with path length
// D = D_c + delta, and the band centre f_c = f0 + k_c df, k_c = (K - 1)/2,
//
//   f_k D = f0 D_c + f_c delta + k df D_c + (k - k_c) df delta,
//
// so the element factors as
//
//   A_kv = p_k amp_v e^{-j 2 pi (f0 D_c + f_c delta_v)/c} e^{-j 2 pi k df D_c/c} e^{-j z_k t_v},
//   t_v = delta_v / xi  (|t_v| <= 0.95 for every voxel slot),  z_k = 2 pi (k - k_c) df xi / c,
//
// and the last factor has the Jacobi-Anger (Chebyshev) expansion
//
//   e^{-j z t} = sum_l (-j)^l b_l(z) T_l(t),   b_0 = J_0(z),  b_l = 2 J_l(z),
//
// truncated after L terms (L even, tail below 2e-6 at the band edges |z| = z_max;
// centring halves z_max and with it the number of terms).  So per (pair, tile)
//
//   forward:  y_k += P_k sum_l (-j)^l b_l(k) m_l,  m_l = sum_v u_v T_l(t_v),
//             u_v = amp_v s_v e^{-j 2 pi (f0 D_c + f_c delta_v)/c},  P_k = e^{-j 2 pi k df D_c/c}
//   adjoint:  g_v += conj(u'_v) sum_l T_l(t_v) C_l,  C_l = j^l sum_k b_l(k) conj(p_k) r_k conj(P_k),
//             u'_v = amp_v e^{-j 2 pi (f0 D_c + f_c delta_v)/c}.
//
// The per-voxel work is L steps of the Chebyshev recurrence T_{l+1} = 2t T_l - T_{l-1}
// (stable for |t| <= 0.95: rounding grows at most 3.2 l times) with two FMAs
// each, instead of K complex terms; the per-(pair, tile) work is 2KL FMAs.
// b_l(k) is real, so each (k, l) term of the expansion is two FMAs.
#include "nfm_kernels.cuh"
#include "cheb_device.cuh"

namespace nfm {

// ---------------------------------------------------------------------------
// forward: CTA = ng = blockDim.x / G groups of G lanes (G = 4 or 8); group = (pair, tile of the
// stage); PCH pairs per CTA and TS = ng / PCH tiles per stage
// ---------------------------------------------------------------------------
// 4-lane groups: 96 registers (5 CTAs of 128 threads per SM); 8-lane groups hold half the voxels
// per lane and are capped at 72 registers (7 CTAs per SM) so nearly twice the warps stay resident.
// The CTA body for pair group pg and voxel-tile chunk `chunk` (the single-scene kernel passes blockIdx.x
// and blockIdx.y; the multi-scene kernel its CTA's position within its scene).
template <int LT, int G, int TZ>
__device__ __forceinline__ void fwd_cheb_body(const OpDesc op, const ChebDesc cd, const FwdArgs a, int pg,
                                              int chunk, unsigned char* smem)
{
    constexpr int TV = TILE_X * TILE_Y * TZ; // voxels of a tile (TZ = TILE_Z) or of a two-tile block (TZ = 8)
    constexpr int LS = (LT + 3) & ~3;        // table row stride (zero entries beyond LT)
    constexpr int LSS = fwd_coef_stride(LT); // its row stride in shared memory
    const int ng = blockDim.x / G;           // groups per CTA
    const int PCH = a.VS;                    // pairs per CTA (power of two dividing ng)
    const int TS = ng / PCH;                 // tiles per stage
    const int K = op.K;
    const int KP = cd.k_pad;                 // table rows (multiple of 4, zero rows beyond K)
    const int AS = KP + 4;                   // accumulator row stride (float2), staggers the banks
    const int CR = fwd_coef_rows(KP);        // table rows held: k <= K/2 (the rest follow by the mirror fold)
    float* coef = reinterpret_cast<float*>(smem);                            // [CR][LSS]
    float2* acc = reinterpret_cast<float2*>(coef + CR * LSS);                // [ng][AS]
    float2* s_st = reinterpret_cast<float2*>(acc + ng * AS);                 // [2][TS][TV]
    AntHead* ant_st = reinterpret_cast<AntHead*>(s_st + 2 * TS * TV);        // [ng][2], one stage
    int* pair_s = reinterpret_cast<int*>(ant_st + ng * 2);                   // [PCH] pair or -1
    // explicit voxel positions: the stage's voxel offsets [2][TS][TILE_V] (16-byte aligned after pair_s)
    VoxelOffset* vox_st = reinterpret_cast<VoxelOffset*>(pair_s + ((PCH + 3) & ~3));

    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    const int g = tid / G, ln = tid % G;
    const int pl = g % PCH, slot = g / PCH;
    const unsigned gmask = ((1u << G) - 1u) << ((tid % 32) & ~(G - 1));
    const int pair_base = pg * PCH;
    const int t_begin = chunk * a.tiles_base + min(chunk, a.tiles_rem);
    const int t_end = t_begin + a.tiles_base + (chunk < a.tiles_rem ? 1 : 0);
    const int n_stages = (t_end - t_begin + TS - 1) / TS;

    // Constants and the pair list: no kernel of this library writes them, so they are read
    // before the wait on the previous kernel (which may still be running its tail).  (Plain loads:
    // asynchronous copies of the table measured slower here.)
    for (int i = tid; i < CR * LS / 4; i += nt)
        reinterpret_cast<float4*>(coef)[(i / (LS / 4)) * (LSS / 4) + i % (LS / 4)] =
            reinterpret_cast<const float4*>(cd.coef)[i];
    const bool pts = TZ == TILE_Z && op.g.pts;   // explicit positions come in 128-voxel tiles only
    for (int i = tid; i < ng * AS / 2; i += nt)   // the per-slot spectra start at zero (AS even)
        reinterpret_cast<float4*>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < PCH) {
        const int sp = pair_base + tid;
        int pair = sp < a.n_pairs ? a.pairs[sp] : -1;
        if (sp < a.n_pairs && (pair < 0 || pair >= op.P)) {   // flagged; pair 0 keeps every access in bounds
            atomicOr(op.err, ERRF_PAIR);
            pair = 0;
        }
        pair_s[tid] = pair;
    }
    __syncthreads();

    auto load_geom = [&](int q) {                 // the leading 32 B of the two antenna-tile rows of every group
        for (int i = tid; i < ng * 4; i += nt) {
            const int gi = i / 4, part = i % 4;
            const int tile = t_begin + q * TS + gi / PCH;
            const int pair = pair_s[gi % PCH];
            if (tile < t_end && pair >= 0) {
                const AntTile *at, *ar;
                pair_rows(op, pair, tile, at, ar);
                AntHead* dst = ant_st + gi * 2 + (part < 2 ? 0 : 1);
                cp_async_16(reinterpret_cast<float4*>(dst) + part % 2,
                            reinterpret_cast<const float4*>(part < 2 ? at : ar) + part % 2);
            }
        }
    };
    // offsets of this thread's voxel slots (tid, and tid + nt when nt < TILE_V) within a tile in the
    // scene vector (grid rows of nx, planes of nx ny); a full tile's values are then one add away from
    // its origin
    const int plane = op.g.nx * op.g.ny;
    auto slot_offset = [&](int v) {
        return (v / (TILE_X * TILE_Y)) * plane + ((v / TILE_X) % TILE_Y) * op.g.nx + v % TILE_X;
    };
    auto load_s = [&](int q) {                    // the stage's scene values (zero outside the grid)
        const int buf = q & 1;
        if (pts) {                                // explicit positions: voxel n = tile * 128 + slot, and its offset
            for (int sl = 0; sl < TS; ++sl) {
                const int tile = t_begin + q * TS + sl;
                if (tile >= t_end) break;
                for (int v = tid; v < TILE_V; v += nt) {
                    const long long n = (long long)tile * TILE_V + v;
                    const bool in = n < op.g.nx;
                    cp_async_8(s_st + (buf * TS + sl) * TILE_V + v, in ? a.s + NFM_IDX(n, op.n_vox, op.err) : a.s, in);
                    cp_async_16(vox_st + (buf * TS + sl) * TILE_V + v, op.g.pts + n);   // padded to whole tiles
                }
            }
            return;
        }
        const int v1 = tid + nt;                  // (computed per call: nothing stays live across stages)
        const int off0 = slot_offset(tid), off1 = v1 < TV ? slot_offset(v1) : 0;
        int tx, ty, tz;                           // coordinates of the stage's first tile, then stepped
        tile_coords(op.g, t_begin + q * TS, tx, ty, tz);
        for (int sl = 0; sl < TS; ++sl) {
            if (t_begin + q * TS + sl >= t_end) break;   // slots past the chunk stay idle
            const int x0 = tx * TILE_X, y0 = ty * TILE_Y, z0 = tz * TZ;
            const bool full = x0 + TILE_X <= op.g.nx && y0 + TILE_Y <= op.g.ny && z0 + TZ <= op.g.nz;
            float2* dst = s_st + (buf * TS + sl) * TV;
            const long long obase = ((long long)z0 * op.g.ny + y0) * op.g.nx + x0;   // index of origin in s
            if (full && 2 * nt >= TV) {           // one or two slots per thread, offsets precomputed
                cp_async_8(dst + tid, a.s + NFM_IDX(obase + off0, op.n_vox, op.err), true);
                if (v1 < TV) cp_async_8(dst + v1, a.s + NFM_IDX(obase + off1, op.n_vox, op.err), true);
            } else if (full) {
                for (int v = tid; v < TV; v += nt)
                    cp_async_8(dst + v, a.s + NFM_IDX(obase + slot_offset(v), op.n_vox, op.err), true);
            } else {
                for (int v = tid; v < TV; v += nt) {
                    const int ix = x0 + v % TILE_X, iy = y0 + (v / TILE_X) % TILE_Y, iz = z0 + v / (TILE_X * TILE_Y);
                    const bool in = ix < op.g.nx && iy < op.g.ny && iz < op.g.nz;
                    cp_async_8(dst + v, in ? a.s + NFM_IDX(obase + slot_offset(v), op.n_vox, op.err) : a.s, in);
                }
            }
            if (++tx == op.g.tiles_x) {           // next tile in x-fastest order
                tx = 0;
                if (++ty == op.g.tiles_y) {
                    ty = 0;
                    ++tz;
                }
            }
        }
    };

    if (n_stages > 0) load_geom(0);
    pdl_wait();                              // s may come from the previous kernel
    if (n_stages > 0) {
        load_s(0);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
    }
    for (int q = 0; q < n_stages; ++q) {
        const int buf = q & 1;
        const int tile = t_begin + q * TS + slot;
        const bool live = tile < t_end && pair_s[pl] >= 0;   // uniform over the group's lanes
        PairTile P;
        if (live) {
            P = fold_pair_head(ant_st[g * 2], ant_st[g * 2 + 1]);
            centre_base_phase(P, K);
        }
        if (q + 1 < n_stages) {
            __syncthreads();                 // every group holds its heads: the buffer takes the next stage's
            load_geom(q + 1);
            load_s(q + 1);
            cp_async_commit();
        }
        if (live) {
            const float2* sb = s_st + (buf * TS + slot) * TV;
            float mr[LT], mi[LT];
#pragma unroll
            for (int l = 0; l < LT; ++l) mr[l] = mi[l] = 0.f;
            // m_l += u_v T_l(t_v), u_v = amp_v s_v e^{-j 2 pi (f0 D_c + f_c delta_v)/c}, t_v = delta_v / xi
            auto add_voxel = [&](const float2 sv, const ChebVoxel& cv) {
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
            };
            if (pts) {
                const VoxelOffset* vsrc = vox_st + (buf * TS + slot) * TILE_V;
#pragma unroll 2
                for (int i = 0; i < TILE_V / G; ++i) {
                    const int v = ln + G * i;
                    add_voxel(sb[v], cheb_voxel(P, vsrc[v], cd.fc_hi, cd.fc_lo));
                }
            } else {
                // On the grid, q = d^2 - d_c^2 = |u|^2 - 2 v.u splits over the axes into the sum of
                // w (w - 2 v_w), w = u_x, u_y, u_z.  The lane's voxels are the columns lx = ln + G a of every
                // row (ly, lz), in x-fastest order: the x terms are formed once per (pair, block), the z terms
                // once per plane and the y terms once per row.
                constexpr int NA = TILE_X / G;
                float xT[NA], xR[NA];
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const float ux = voxel_offset(op.g, ln + G * a, 0, 0, TZ).ux;
                    xT[a] = ux * fmaf(-2.f, P.vTx, ux);
                    xR[a] = ux * fmaf(-2.f, P.vRx, ux);
                }
#pragma unroll 1
                for (int lz = 0; lz < TZ; ++lz) {
                    const float uz = voxel_offset(op.g, 0, 0, lz, TZ).uz;
                    const float zT = uz * fmaf(-2.f, P.vTz, uz), zR = uz * fmaf(-2.f, P.vRz, uz);
#pragma unroll
                    for (int ly = 0; ly < TILE_Y; ++ly) {
                        const float uy = voxel_offset(op.g, 0, ly, 0, TZ).uy;
                        const float yzT = fmaf(uy, fmaf(-2.f, P.vTy, uy), zT);
                        const float yzR = fmaf(uy, fmaf(-2.f, P.vRy, uy), zR);
#pragma unroll
                        for (int a = 0; a < NA; ++a) {
                            const int v = ln + G * a + TILE_X * (ly + TILE_Y * lz);
                            add_voxel(sb[v], cheb_voxel_q(P, xT[a] + yzT, xR[a] + yzR, cd.fc_hi, cd.fc_lo));
                        }
                    }
                }
            }
            // all-reduce over the group's lanes (the same sum order in every lane)
#pragma unroll
            for (int w = 1; w < G; w *= 2) {
#pragma unroll
                for (int l = 0; l < LT; ++l) {
                    mr[l] += __shfl_xor_sync(gmask, mr[l], w);
                    mi[l] += __shfl_xor_sync(gmask, mi[l], w);
                }
            }
            // expansion over half the band: the band-centred table is mirror-symmetric,
            // b_l(K-1-k) = (-1)^l b_l(k), so with E = sum over even l and O = sum over odd l of
            // (-j)^l b_l(k) m_l, S_k = E + O and S_{K-1-k} = E - O.  Lane ln owns k = ln + G j < K/2 and the
            // mirrors; (-j)^l is applied by permuting re/im.  The tile phasors run from the band centre (the
            // base phase carries e^{-j 2 pi k_c S}, S = df D_c/c): k takes conj(c), c = e^{+j 2 pi (k - k_c) S},
            // and its mirror K-1-k takes c, one phasor per k-pair advanced by W = e^{+j 2 pi G S} (Taylor
            // phasor, error ~1e-7, at most K/(2G) steps) from a directly evaluated start; for odd K one lane
            // adds the centre row (phasor 1).
            float2* accg = acc + g * AS;
            const int KH = K / 2;
            float2 cu = tile_step_cis_f(P, (float)ln - 0.5f * (float)(K - 1));
            const float2 W = tile_step_cis_exact(P, G);
            auto accumulate = [&](int k, float2 c, float sr, float si) {   // y_k += P_k S_k, P_k = (c.x, -c.y)
                float2 av = accg[k];
                av.x = fmaf(c.x, sr, fmaf(c.y, si, av.x));
                av.y = fmaf(c.x, si, fmaf(-c.y, sr, av.y));
                accg[k] = av;
            };
            for (int k = ln; k < KH; k += G) {
                const float* b0 = coef + k * LSS;
                float er = 0.f, ei = 0.f, orr = 0.f, oi = 0.f;
#pragma unroll
                for (int l = 0; l < LT; l += 4) {
                    const float4 x = *reinterpret_cast<const float4*>(b0 + l);
                    er = fmaf(x.x, mr[l], er);
                    ei = fmaf(x.x, mi[l], ei);
                    orr = fmaf(x.y, mi[l + 1], orr);
                    oi = fmaf(-x.y, mr[l + 1], oi);
                    if (l + 2 < LT) {                    // LT is even: l + 2 < LT covers l + 3
                        er = fmaf(-x.z, mr[l + 2], er);
                        ei = fmaf(-x.z, mi[l + 2], ei);
                        orr = fmaf(-x.w, mi[l + 3], orr);
                        oi = fmaf(x.w, mr[l + 3], oi);
                    }
                }
                accumulate(k, cu, er + orr, ei + oi);
                accumulate(K - 1 - k, make_float2(cu.x, -cu.y), er - orr, ei - oi);
                cu = cmul(cu, W);
            }
            if ((K & 1) && ln == KH % G) {               // centre row k_c = K/2 (its own mirror)
                const float* b0 = coef + KH * LSS;
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int l = 0; l < LT; l += 4) {
                    const float4 x = *reinterpret_cast<const float4*>(b0 + l);
                    sr = fmaf(x.x, mr[l], sr);
                    si = fmaf(x.x, mi[l], si);
                    sr = fmaf(x.y, mi[l + 1], sr);
                    si = fmaf(-x.y, mr[l + 1], si);
                    if (l + 2 < LT) {
                        sr = fmaf(-x.z, mr[l + 2], sr);
                        si = fmaf(-x.z, mi[l + 2], si);
                        sr = fmaf(-x.w, mi[l + 3], sr);
                        si = fmaf(x.w, mr[l + 3], si);
                    }
                }
                accumulate(KH, make_float2(1.f, 0.f), sr, si);
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
    pdl_launch_dependents();

    // sum the live stage slots of each pair in slot order and write the chunk partial (the rows start
    // at zero and every live slot added its tiles); the threads split as (nt / K) pairs x K
    // frequencies when K <= nt
    const int live_slots = min(TS, t_end - t_begin);
    const bool kfit = K <= nt;
    const int p_step = kfit ? nt / K : 1;
    const int p_first = kfit ? (tid / K < p_step ? tid / K : PCH) : 0;
    const int k_first = kfit ? tid % K : tid, k_step = kfit ? K : nt;
    for (int p = p_first; p < PCH; p += p_step) {
        const int sp = pair_base + p;
        if (sp >= a.n_pairs) break;
        const long long out0 = ((long long)chunk * a.n_slots + sp) * K;
        float2* out = a.partial + out0;
        for (int k = k_first; k < K; k += k_step) {
            const float2* col = acc + p * AS + k;
            float2 sum = col[0];
#pragma unroll 4
            for (int sl = 1; sl < live_slots; ++sl) {
                const float2 x = col[sl * PCH * AS];
                sum.x += x.x;
                sum.y += x.y;
            }
#ifdef NFM_BOUNDS_CHECK
            a.partial[NFM_IDX(out0 + k, a.partial_elems, op.err)] = sum;
#else
            out[k] = sum;
#endif
        }
    }
}

template <int LT, int G, int TZ>
__global__ void __launch_bounds__(CHEB_THREADS, G == 8 ? 7 : 5) fwd_cheb_kernel(OpDesc op, ChebDesc cd, FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    fwd_cheb_body<LT, G, TZ>(op, cd, a, blockIdx.x, blockIdx.y, smem);
}

// ---------------------------------------------------------------------------
// adjoint: CTA = one block of 8 x 4 x TZ voxels, thread = voxel; pairs in chunks of adj_cheb_pchunk(TZ).
// TZ = 4: the tiles of the geometry (TILE_V voxels); TZ = 8: blocks of two tiles along z, with their own
// antenna-block table and expansion table (op.g, op.ant and cd describe the blocks), which halves the
// per-voxel share of the per-(pair, block) work: the residual transform and the coefficient stage.
// ---------------------------------------------------------------------------
template <int LT, int TZ>
__device__ __forceinline__ void adj_cheb_body(const OpDesc op, const ChebDesc cd, const AdjArgs a, int tile,
                                              unsigned char* smem)
{
    constexpr int LS = (LT + 3) & ~3;        // table row stride (zero entries beyond LT)
    constexpr int TV = TILE_X * TILE_Y * TZ; // voxels of a block = threads of the CTA
    constexpr int PCH = adj_cheb_pchunk(TZ); // pairs staged per round
    const int K = op.K;
    const int KP = cd.k_pad;
    float* coef = reinterpret_cast<float*>(smem);                          // [KP][LS]
    const int RS = KP + 2;                   // r' row stride (float2), staggers the banks
    float2* rp = reinterpret_cast<float2*>(coef + KP * LS);               // [PCH][RS]
    float2* Cs = rp + PCH * RS;                                             // [PCH][LS]
    PairTile* pt = reinterpret_cast<PairTile*>(Cs + PCH * LS);              // [PCH], as pair_tile_adj leaves them
    float2* w16 = reinterpret_cast<float2*>(pt + PCH);                      // [PCH] e^{+j 2 pi 16 df D_c/c}

    const int tid = threadIdx.x;
    int tx, ty, tz;
    tile_coords(op.g, tile, tx, ty, tz);
    const int lx = tid % TILE_X, ly = (tid / TILE_X) % TILE_Y, lz = tid / (TILE_X * TILE_Y);
    VoxelOffset o;
    if (TZ == TILE_Z && op.g.pts) {          // explicit positions: voxel n = tile * 128 + thread
        const float4 u = op.g.pts[(size_t)tile * TILE_V + tid];
        o.ux = u.x;
        o.uy = u.y;
        o.uz = u.z;
        o.uu = u.w;
    } else {
        o = voxel_offset(op.g, lx, ly, lz, TZ);
    }
    for (int i = tid; i < KP * LS / 4; i += TV)
        reinterpret_cast<float4*>(coef)[i] = reinterpret_cast<const float4*>(cd.coef)[i];
    constexpr int LQ = LS / 4;
    float gr = 0.f, gi = 0.f;
    // the pair list and the geometry tables are never written by this library's kernels, so the
    // first chunk's pair tiles are read before the wait on the previous kernel
    if (tid < min(PCH, a.n_pairs)) {
        pt[tid] = pair_tile_adj(load_pair_tile(op, a.pairs[tid], tile), K);
        w16[tid] = tile_step_cis_exact(pt[tid], 16);
    }
    pdl_wait();                              // r comes from the previous kernel
    // the voxel's iterate for the fused update, loaded now so that its latency overlaps the r copies
    const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TZ + lz;
    const size_t np = (size_t)tile * TILE_V + tid;
    const bool pts = TZ == TILE_Z && op.g.pts;
    const bool in_grid = pts ? np < (size_t)op.g.nx : (ix < op.g.nx && iy < op.g.ny && iz < op.g.nz);
    const size_t n = !in_grid ? 0 : pts ? np : ((size_t)iz * op.g.ny + iy) * op.g.nx + ix;
    const float2 s_old = (a.s && in_grid) ? a.s[NFM_IDX(n, op.n_vox, op.err)] : make_float2(0.f, 0.f);

    // rows of r start on 16-byte boundaries in shared memory (RS even) and, for even K, in r
    const bool r_vec = !(K & 1) && !(reinterpret_cast<uintptr_t>(a.r) & 15);
    for (int c0 = 0; c0 < a.n_pairs; c0 += PCH) {
        const int nc = min(PCH, a.n_pairs - c0);
        if (c0 > 0) {
            __syncthreads();
            if (tid < nc) {
                pt[tid] = pair_tile_adj(load_pair_tile(op, a.pairs[c0 + tid], tile), K);
                w16[tid] = tile_step_cis_exact(pt[tid], 16);
            }
        }
        // The chunk's residual rows into rp, 16 threads per pair: every thread issues all its copies before
        // it waits, so the loads overlap (one L2 round trip).
        const int k0 = tid % 16;
        if (r_vec) {                         // 16-byte copies of (r_k, r_k+1), k even (K even, r 16-byte aligned)
            for (int j = tid / 16; j < nc; j += TV / 16)
                for (int k = 2 * k0; k < K; k += 32)
                    cp_async_16_ca(rp + j * RS + k, a.r + NFM_IDX((long long)(c0 + j) * K + k, a.r_elems, op.err));
        } else {
            for (int j = tid / 16; j < nc; j += TV / 16)
                for (int k = k0; k < K; k += 16)
                    cp_async_8(rp + j * RS + k, a.r + NFM_IDX((long long)(c0 + j) * K + k, a.r_elems, op.err), true);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();                     // pt and w16 of this chunk
        // r'_k = conj(p_k) r_k e^{+j 2 pi (k - k_c) S}, S = df D_c/c, for k and its mirror K-1-k, folded in place into
        // u_k = r'_k + r'_{K-1-k} (stored at k) and v_k = r'_k - r'_{K-1-k} (stored at K-1-k), k < K/2; for odd K
        // the centre row k_c = K/2 keeps r'.  The band-centred table is mirror-symmetric,
        // b_l(K-1-k) = (-1)^l b_l(k), so C_l needs only b_l(k) u_k (even l) and b_l(k) v_k (odd l) over half the
        // band.  A thread owns both slots of its k, so no barrier separates the transform from the fold.
        // Phasors run from the band centre (the pair tile's base phase carries e^{+j 2 pi k_c S}): k takes
        // c = e^{+j 2 pi (k - k_c) S} and its mirror K-1-k the conjugate, so with A = x + y, B = x - y
        //   u = x c + y conj(c) = (c_r A_r - c_i B_i, c_r A_i + c_i B_r),
        //   v = x c - y conj(c) = (c_r B_r - c_i A_i, c_r B_i + c_i A_r).
        // c starts from an SFU phasor at k0 and steps by the pair's exact 16-step phasor (at most 4 steps);
        // the centre row of odd K takes c = 1.
        const int KH = K / 2;
        const float kc = 0.5f * (float)(K - 1);
        for (int j = tid / 16; j < nc; j += TV / 16) {
            const float2 W = w16[j];
            float2* row = rp + j * RS;
            float2 c = tile_step_cis_f(pt[j], (float)k0 - kc);
            for (int k = k0; k < KH; k += 16) {
                const int km = K - 1 - k;
                float2 x = row[k], y = row[km];
                if (op.pulse) {
                    x = cmul_conj(x, op.pulse[k]);
                    y = cmul_conj(y, op.pulse[km]);
                }
                const float Ar = x.x + y.x, Ai = x.y + y.y, Br = x.x - y.x, Bi = x.y - y.y;
                row[k] = make_float2(fmaf(c.x, Ar, -c.y * Bi), fmaf(c.x, Ai, c.y * Br));
                row[km] = make_float2(fmaf(c.x, Br, -c.y * Ai), fmaf(c.x, Bi, c.y * Ar));
                c = cmul(c, W);
            }
            if ((K & 1) && op.pulse && k0 == KH % 16) row[KH] = cmul_conj(row[KH], op.pulse[KH]);   // centre row
        }
        __syncthreads();
        // C_l = j^l sum_k b_l(k) r'_k = j^l [sum_{k < K/2} b_l(k) (u_k or v_k) + b_l(k_c) r'_{k_c}], four l per task,
        // each task split over the parity of k between lanes e and e ^ 1 (combined by one shuffle; the pair's
        // rows and table rows of the two parities sit in different banks); the centre row goes to parity 0
        {
            const int n_task = 2 * nc * LQ;  // even, so lane pairs never straddle a round or the end
            for (int e0 = 0; e0 < n_task; e0 += TV) {
                const int e = e0 + tid;
                const bool active = e < n_task;
                if (!__any_sync(0xffffffffu, active)) continue;   // whole warp past the end
                const int h = e & 1, et = (active ? e : 0) >> 1;
                const int j = et / LQ, l = 4 * (et - (et / LQ) * LQ);
                const float2* rj = rp + j * RS;
                float cr0 = 0.f, ci0 = 0.f, cr1 = 0.f, ci1 = 0.f, cr2 = 0.f, ci2 = 0.f, cr3 = 0.f, ci3 = 0.f;
                for (int k = active ? h : KH; k < KH; k += 2) {
                    const float2 u = rj[k], v = rj[K - 1 - k];
                    const float4 b = *reinterpret_cast<const float4*>(coef + k * LS + l);
                    cr0 = fmaf(b.x, u.x, cr0);
                    ci0 = fmaf(b.x, u.y, ci0);
                    cr1 = fmaf(b.y, v.x, cr1);
                    ci1 = fmaf(b.y, v.y, ci1);
                    cr2 = fmaf(b.z, u.x, cr2);
                    ci2 = fmaf(b.z, u.y, ci2);
                    cr3 = fmaf(b.w, v.x, cr3);
                    ci3 = fmaf(b.w, v.y, ci3);
                }
                if ((K & 1) && active && h == 0) {   // the centre row (b_l(k_c), l >= 1, is zero up to rounding)
                    const float2 w = rj[KH];
                    const float4 b = *reinterpret_cast<const float4*>(coef + KH * LS + l);
                    cr0 = fmaf(b.x, w.x, cr0);
                    ci0 = fmaf(b.x, w.y, ci0);
                    cr1 = fmaf(b.y, w.x, cr1);
                    ci1 = fmaf(b.y, w.y, ci1);
                    cr2 = fmaf(b.z, w.x, cr2);
                    ci2 = fmaf(b.z, w.y, ci2);
                    cr3 = fmaf(b.w, w.x, cr3);
                    ci3 = fmaf(b.w, w.y, ci3);
                }
                cr0 += __shfl_xor_sync(0xffffffffu, cr0, 1);
                ci0 += __shfl_xor_sync(0xffffffffu, ci0, 1);
                cr1 += __shfl_xor_sync(0xffffffffu, cr1, 1);
                ci1 += __shfl_xor_sync(0xffffffffu, ci1, 1);
                cr2 += __shfl_xor_sync(0xffffffffu, cr2, 1);
                ci2 += __shfl_xor_sync(0xffffffffu, ci2, 1);
                cr3 += __shfl_xor_sync(0xffffffffu, cr3, 1);
                ci3 += __shfl_xor_sync(0xffffffffu, ci3, 1);
                if (active && h == 0) {
                    float2* Cj = Cs + j * LS + l;  // l % 4 == 0: factors 1, j, -1, -j
                    Cj[0] = make_float2(cr0, ci0);
                    Cj[1] = make_float2(-ci1, cr1);
                    Cj[2] = make_float2(-cr2, -ci2);
                    Cj[3] = make_float2(ci3, -cr3);
                }
            }
        }
        __syncthreads();
        // per voxel: sum over the chunk's pairs of conj(u') sum_l T_l(t) C_l; the geometry of pair
        // j+1 is computed next to the recurrence of pair j (independent instructions)
        auto stage_pair = [&](int j, float2& w, float& t) {
            const ChebVoxel cv = cheb_voxel_m2(pt[j], o, cd.fc_hi, cd.fc_lo);
            const float2 c0v = cis_turns_sfu(cv.th0);
            w = make_float2(cv.amp * c0v.x, cv.amp * c0v.y);
            t = cv.delta * cd.tau;
        };
        float2 w;
        float t;
        // pair j's coefficient sum and its contribution to g (the coefficients are read into registers
        // first, so the recurrence does not wait on shared-memory latency term by term)
        auto add_pair = [&](int j, float2 wj, float tj) {
            const float t2 = tj + tj;
            const float4* C = reinterpret_cast<const float4*>(Cs + j * LS);
            float4 cr[LT / 2];
#pragma unroll
            for (int i = 0; i < LT / 2; ++i) cr[i] = C[i];
            float4 q = cr[0];
            float ar = fmaf(tj, q.z, q.x), ai = fmaf(tj, q.w, q.y);
            float Tp = 1.f, Tc = tj;
#pragma unroll
            for (int l = 2; l < LT; l += 2) {
                q = cr[l / 2];
                const float Ta = fmaf(t2, Tc, -Tp);
                const float Tb = fmaf(t2, Ta, -Tc);
                ar = fmaf(Ta, q.x, ar);
                ai = fmaf(Ta, q.y, ai);
                ar = fmaf(Tb, q.z, ar);
                ai = fmaf(Tb, q.w, ai);
                Tp = Ta;
                Tc = Tb;
            }
            gr = fmaf(wj.x, ar, fmaf(-wj.y, ai, gr));
            gi = fmaf(wj.x, ai, fmaf(wj.y, ar, gi));
        };
        stage_pair(0, w, t);
#pragma unroll 2
        for (int j = 0; j + 1 < nc; ++j) {   // the last pair is peeled: nothing left to stage
            float2 wn;
            float tn;
            stage_pair(j + 1, wn, tn);
            add_pair(j, w, t);
            w = wn;
            t = tn;
        }
        add_pair(nc - 1, w, t);
    }
    pdl_launch_dependents();

    if (a.s) {                               // every lane takes part (group norms use the warp)
        const float2 out = step_prox(s_old, gr, gi, a.step, a.alpha, a.alpha_g, a.shrink, in_grid);
        if (in_grid) a.s[NFM_IDX(n, op.n_vox, op.err)] = out;
    } else if (in_grid) {
        a.g_out[NFM_IDX(n, op.n_vox, op.err)] = make_float2(gr, gi);
    }
}

// at most 64 registers either way: 8 CTAs of 128 threads or 4 of 256 per SM
template <int LT, int TZ>
__global__ void __launch_bounds__(TILE_X * TILE_Y * TZ, TZ == TILE_Z ? 8 : 4) adj_cheb_kernel(OpDesc op, ChebDesc cd,
                                                                                         AdjArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    adj_cheb_body<LT, TZ>(op, cd, a, blockIdx.x, smem);
}

// ---------------------------------------------------------------------------
// the same bodies over several scenes in one launch (batched SPGM): the CTA finds its scene item
// ---------------------------------------------------------------------------
template <typename Item>
__device__ __forceinline__ int multi_item(const Item* __restrict__ items, int n_items)
{
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].cta0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int LT>
__global__ void __launch_bounds__(CHEB_THREADS, 5) fwd_cheb_multi_kernel(const MultiFwdItem* __restrict__ items,
                                                                         int n_items)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int i = multi_item(items, n_items);
    const OpDesc op = items[i].op;
    const ChebDesc cd = items[i].cd;
    const FwdArgs a = items[i].a;
    const int local = (int)blockIdx.x - items[i].cta0, ng = items[i].n_groups;
    fwd_cheb_body<LT, CHEB_GROUP, TILE_Z>(op, cd, a, local % ng, local / ng, smem);
}

template <int LT>
__global__ void __launch_bounds__(CHEB_THREADS, 7) adj_cheb_multi_kernel(const MultiAdjItem* __restrict__ items,
                                                                         int n_items)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int i = multi_item(items, n_items);
    const OpDesc op = items[i].op;
    const ChebDesc cd = items[i].cd;
    const AdjArgs a = items[i].a;
    adj_cheb_body<LT, TILE_Z>(op, cd, a, (int)blockIdx.x - items[i].cta0, smem);
}

// ---------------------------------------------------------------------------
// FP64 range of delta: max over antennas, tiles and the 128 voxel slots of each
// tile (including slots beyond the grid edge) of | |r_a - r_v| - |r_a - r_c| |
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) cheb_range_kernel(GridDesc g, AntSetup a, unsigned long long* out)
{
    __shared__ double red[256];
    double mx = 0.0;
    const long long total = (long long)a.n_ant * g.n_tiles;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ant = (int)(i / g.n_tiles);
        const int tile = (int)(i - (long long)ant * g.n_tiles);
        const double ax = a.ant_xyz[3 * ant], ay = a.ant_xyz[3 * ant + 1], az = a.ant_xyz[3 * ant + 2];
        if (a.tile_c) {                      // explicit voxel positions: the tile's voxels about its centre
            const double cx = a.tile_c[3 * (size_t)tile], cy = a.tile_c[3 * (size_t)tile + 1],
                         cz = a.tile_c[3 * (size_t)tile + 2];
            const double dc = sqrt((ax - cx) * (ax - cx) + (ay - cy) * (ay - cy) + (az - cz) * (az - cz));
            for (int v = 0; v < TILE_V; ++v) {
                const long long n = (long long)tile * TILE_V + v;
                if (n >= a.n_vox) break;
                const double* p = a.vox_xyz + 3 * n;
                const double d = sqrt((ax - p[0]) * (ax - p[0]) + (ay - p[1]) * (ay - p[1]) + (az - p[2]) * (az - p[2]));
                mx = fmax(mx, fabs(d - dc));
            }
            continue;
        }
        int tx, ty, tz;
        tile_coords(g, tile, tx, ty, tz);
        const double cx = a.x0 + (tx * TILE_X + 0.5 * (TILE_X - 1)) * a.dx;
        const double cy = a.y0 + (ty * TILE_Y + 0.5 * (TILE_Y - 1)) * a.dy;
        const double cz = a.z0 + (tz * TILE_Z + 0.5 * (TILE_Z - 1)) * a.dz;
        const double dc = sqrt((ax - cx) * (ax - cx) + (ay - cy) * (ay - cy) + (az - cz) * (az - cz));
        for (int v = 0; v < TILE_V; ++v) {
            const double px = a.x0 + (tx * TILE_X + v % TILE_X) * a.dx;
            const double py = a.y0 + (ty * TILE_Y + (v / TILE_X) % TILE_Y) * a.dy;
            const double pz = a.z0 + (tz * TILE_Z + v / (TILE_X * TILE_Y)) * a.dz;
            const double d = sqrt((ax - px) * (ax - px) + (ay - py) * (ay - py) + (az - pz) * (az - pz));
            mx = fmax(mx, fabs(d - dc));
        }
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    // non-negative doubles order like their bit patterns
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t fwd_cheb_smem_bytes(int LT, int k_pad, int pch, int threads, int group, bool points, int tz)
{
    const int ng = threads / group;
    const int TS = ng / pch;
    const int TV = TILE_X * TILE_Y * tz;
    return (size_t)fwd_coef_rows(k_pad) * fwd_coef_stride(LT) * sizeof(float) +
           (size_t)ng * (k_pad + 4) * sizeof(float2) +
           (size_t)2 * TS * TV * sizeof(float2) + (size_t)ng * 2 * sizeof(AntHead) +
           (size_t)((pch + 3) & ~3) * sizeof(int) +
           (points ? (size_t)2 * TS * TILE_V * sizeof(VoxelOffset) : 0);
}

size_t adj_cheb_smem_bytes(int LT, int k_pad, int tz)
{
    const int LS = (LT + 3) & ~3;
    const int pch = adj_cheb_pchunk(tz);
    return (size_t)k_pad * LS * sizeof(float) + (size_t)pch * (k_pad + 2) * sizeof(float2) +
           (size_t)pch * LS * sizeof(float2) + (size_t)pch * sizeof(PairTile) + (size_t)pch * sizeof(float2);
}

template <int G, int TZ>
const void* fwd_cheb_ptr_g(int LT)
{
    switch (LT) {
    case 10: return (const void*)fwd_cheb_kernel<10, G, TZ>;
    case 12: return (const void*)fwd_cheb_kernel<12, G, TZ>;
    case 14: return (const void*)fwd_cheb_kernel<14, G, TZ>;
    case 16: return (const void*)fwd_cheb_kernel<16, G, TZ>;
    case 18: return (const void*)fwd_cheb_kernel<18, G, TZ>;
    case 20: return (const void*)fwd_cheb_kernel<20, G, TZ>;
    case 22: return (const void*)fwd_cheb_kernel<22, G, TZ>;
    case 24: return (const void*)fwd_cheb_kernel<24, G, TZ>;
    default: break;
    }
    if (TZ != TILE_Z) return nullptr;        // the two-tile blocks are built for L <= 24
    switch (LT) {
    case 26: return (const void*)fwd_cheb_kernel<26, G, TILE_Z>;
    case 28: return (const void*)fwd_cheb_kernel<28, G, TILE_Z>;
    case 30: return (const void*)fwd_cheb_kernel<30, G, TILE_Z>;
    case 32: return (const void*)fwd_cheb_kernel<32, G, TILE_Z>;
    default: return nullptr;
    }
}

const void* fwd_cheb_kernel_ptr(int LT, int group, int tz)
{
    if (tz == TILE_Z) return group == 4 ? fwd_cheb_ptr_g<4, TILE_Z>(LT) : group == 8 ? fwd_cheb_ptr_g<8, TILE_Z>(LT) : nullptr;
    if (tz == 2 * TILE_Z)
        return group == 4 ? fwd_cheb_ptr_g<4, 2 * TILE_Z>(LT) : group == 8 ? fwd_cheb_ptr_g<8, 2 * TILE_Z>(LT) : nullptr;
    return nullptr;
}

template <int TZ>
static const void* adj_cheb_ptr_tz(int LT)
{
    switch (LT) {
    case 10: return (const void*)adj_cheb_kernel<10, TZ>;
    case 12: return (const void*)adj_cheb_kernel<12, TZ>;
    case 14: return (const void*)adj_cheb_kernel<14, TZ>;
    case 16: return (const void*)adj_cheb_kernel<16, TZ>;
    case 18: return (const void*)adj_cheb_kernel<18, TZ>;
    case 20: return (const void*)adj_cheb_kernel<20, TZ>;
    case 22: return (const void*)adj_cheb_kernel<22, TZ>;
    case 24: return (const void*)adj_cheb_kernel<24, TZ>;
    default: break;
    }
    if (TZ != TILE_Z) return nullptr;        // the two-tile blocks are built for L <= 24
    switch (LT) {
    case 26: return (const void*)adj_cheb_kernel<26, TILE_Z>;
    case 28: return (const void*)adj_cheb_kernel<28, TILE_Z>;
    case 30: return (const void*)adj_cheb_kernel<30, TILE_Z>;
    case 32: return (const void*)adj_cheb_kernel<32, TILE_Z>;
    default: return nullptr;
    }
}

const void* adj_cheb_kernel_ptr(int LT, int tz)
{
    return tz == TILE_Z ? adj_cheb_ptr_tz<TILE_Z>(LT) : tz == 2 * TILE_Z ? adj_cheb_ptr_tz<2 * TILE_Z>(LT) : nullptr;
}

cudaError_t launch_fwd_cheb(const OpDesc& op, const ChebDesc& cd, const FwdArgs& a, dim3 grid, int threads,
                            int group, int tz, size_t smem, cudaStream_t st)
{
    const void* fn = fwd_cheb_kernel_ptr(cd.L, group, tz);
    if (!fn || (threads != 64 && threads != 128)) return cudaErrorInvalidValue;
    if (a.VS < 1 || (threads / group) % a.VS != 0) return cudaErrorInvalidValue;
    void* args[] = {(void*)&op, (void*)&cd, (void*)&a};
    return launch_pdl(fn, grid, dim3(threads), smem, st, args);
}

cudaError_t launch_adj_cheb(const OpDesc& op, const ChebDesc& cd, const AdjArgs& a, int tz, size_t smem,
                            cudaStream_t st)
{
    const void* fn = adj_cheb_kernel_ptr(cd.L, tz);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&op, (void*)&cd, (void*)&a};
    return launch_pdl(fn, dim3(op.g.n_tiles), dim3(TILE_X * TILE_Y * tz), smem, st, args);
}

const void* fwd_cheb_multi_ptr(int LT)
{
    switch (LT) {
    case 10: return (const void*)fwd_cheb_multi_kernel<10>;
    case 12: return (const void*)fwd_cheb_multi_kernel<12>;
    case 14: return (const void*)fwd_cheb_multi_kernel<14>;
    case 16: return (const void*)fwd_cheb_multi_kernel<16>;
    case 18: return (const void*)fwd_cheb_multi_kernel<18>;
    case 20: return (const void*)fwd_cheb_multi_kernel<20>;
    default: return nullptr;   // the batched launch covers expansion lengths up to 20
    }
}

const void* adj_cheb_multi_ptr(int LT)
{
    switch (LT) {
    case 10: return (const void*)adj_cheb_multi_kernel<10>;
    case 12: return (const void*)adj_cheb_multi_kernel<12>;
    case 14: return (const void*)adj_cheb_multi_kernel<14>;
    case 16: return (const void*)adj_cheb_multi_kernel<16>;
    case 18: return (const void*)adj_cheb_multi_kernel<18>;
    case 20: return (const void*)adj_cheb_multi_kernel<20>;
    default: return nullptr;
    }
}

cudaError_t launch_fwd_cheb_multi(int LT, const MultiFwdItem* items, int n_items, int n_ctas, size_t smem,
                                  cudaStream_t st)
{
    const void* fn = fwd_cheb_multi_ptr(LT);
    if (!fn || n_items < 1 || n_ctas < 1) return cudaErrorInvalidValue;
    void* args[] = {(void*)&items, (void*)&n_items};
    return launch_pdl(fn, dim3(n_ctas), dim3(CHEB_THREADS), smem, st, args);
}

cudaError_t launch_adj_cheb_multi(int LT, const MultiAdjItem* items, int n_items, int n_ctas, size_t smem,
                                  cudaStream_t st)
{
    const void* fn = adj_cheb_multi_ptr(LT);
    if (!fn || n_items < 1 || n_ctas < 1) return cudaErrorInvalidValue;
    void* args[] = {(void*)&items, (void*)&n_items};
    return launch_pdl(fn, dim3(n_ctas), dim3(CHEB_THREADS), smem, st, args);
}

cudaError_t launch_cheb_range(const GridDesc& g, const AntSetup& a, unsigned long long* out, cudaStream_t st)
{
    long long total = (long long)a.n_ant * g.n_tiles;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    cheb_range_kernel<<<blocks, 256, 0, st>>>(g, a, out);
    return cudaGetLastError();
}

}  // namespace nfm
