// Gradient step + complex soft-threshold as a stand-alone differentiable op
// (Eq. 5), for unrolled SPGM, with the elastic-net scaling of the prox:
//
//     z = s - step * g,   out = shrink prox_alpha(z),  prox_alpha(z) = z (1 - alpha/|z|) if |z| > alpha else 0
//
// (shrink = 1 / (1 + eta lambda w2) for R = w1 ||s||_1 + (w2/2) ||s||^2; shrink = 1 is the paper's l1).
//
// The backward kernel uses PyTorch's convention for complex gradients of a
// real loss (grad = dL/dRe + j dL/dIm, i.e. real 2-vectors).  For |z| > alpha
// the real Jacobian of prox is  J = s I + (alpha/r^3) z z^T  (r = |z|,
// s = 1 - alpha/r), which is symmetric, so grad_z = s o + (alpha/r^3)(z.o) z
// with o the incoming gradient; d out/d alpha = -z/r.  For |z| <= alpha the
// output is 0 and every derivative is 0.  The scaling enters as o -> shrink o, and
// d out/d shrink = prox_alpha(z).
#include "nfm_kernels.cuh"

#include <cstdint>

namespace nfm {

__device__ __forceinline__ float2 prox_one(float2 sv, float2 gv, float step, float alpha, float shrink)
{
    const float zr = fmaf(-step, gv.x, sv.x), zi = fmaf(-step, gv.y, sv.y);
    const float mag = sqrtf(zr * zr + zi * zi);
    float2 o = make_float2(0.f, 0.f);
    if (mag > alpha) {
        const float sc = (1.0f - alpha / mag) * shrink;
        o = make_float2(zr * sc, zi * sc);
    }
    return o;
}

__global__ void prox_step_kernel(const float2* s, const float2* g, float step, float alpha, float shrink, long long n,
                                 float2* out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = prox_one(s[i], g[i], step, alpha, shrink);
}

// The same with 16-byte accesses (two elements per load) for 16-byte aligned vectors: an HBM-bound
// stream of 24 bytes per element (read s and g, write out).
__global__ void prox_step_vec_kernel(const float4* s, const float4* g, float step, float alpha, float shrink,
                                     long long n2, float4* out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        const float4 sv = s[i], gv = g[i];
        const float2 a = prox_one(make_float2(sv.x, sv.y), make_float2(gv.x, gv.y), step, alpha, shrink);
        const float2 b = prox_one(make_float2(sv.z, sv.w), make_float2(gv.z, gv.w), step, alpha, shrink);
        out[i] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// grad_s = grad_z, grad_g = -step grad_z, and FP64 block partials of
// d/dstep = -sum grad_z . g, d/dalpha = -shrink sum_{|z|>alpha} (z . o) / |z| and
// d/dshrink = sum o . prox_alpha(z).
__global__ void __launch_bounds__(256) prox_step_backward_kernel(const float2* s, const float2* g, float step,
                                                                 float alpha, float shrink, long long n,
                                                                 const float2* go, float2* grad_s, float2* grad_g,
                                                                 double* partial)
{
    __shared__ double sh0[256], sh1[256], sh2[256];
    double a_step = 0.0, a_alpha = 0.0, a_shrink = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float2 sv = s[i], gv = g[i], o0 = go[i];
        const float2 o = make_float2(shrink * o0.x, shrink * o0.y);
        const float zr = fmaf(-step, gv.x, sv.x), zi = fmaf(-step, gv.y, sv.y);
        const float mag = sqrtf(zr * zr + zi * zi);
        float2 gz = make_float2(0.f, 0.f);
        if (mag > alpha) {
            const float sc = 1.0f - alpha / mag;
            const float zo = zr * o.x + zi * o.y;
            const float k = alpha / (mag * mag * mag) * zo;
            gz = make_float2(fmaf(sc, o.x, k * zr), fmaf(sc, o.y, k * zi));
            a_alpha -= (double)zo / (double)mag;
            a_shrink += (double)sc * ((double)zr * o0.x + (double)zi * o0.y);
        }
        if (grad_s) grad_s[i] = gz;
        if (grad_g) grad_g[i] = make_float2(-step * gz.x, -step * gz.y);
        a_step -= (double)gz.x * gv.x + (double)gz.y * gv.y;
    }
    sh0[threadIdx.x] = a_step;
    sh1[threadIdx.x] = a_alpha;
    sh2[threadIdx.x] = a_shrink;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh0[threadIdx.x] += sh0[threadIdx.x + w];
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
            sh2[threadIdx.x] += sh2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[3 * blockIdx.x] = sh0[0];
        partial[3 * blockIdx.x + 1] = sh1[0];
        partial[3 * blockIdx.x + 2] = sh2[0];
    }
}

__global__ void sum_triples_kernel(const double* partial, int nb, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < nb; ++i) {
            a += partial[3 * i];
            b += partial[3 * i + 1];
            c += partial[3 * i + 2];
        }
        out[0] = a;
        out[1] = b;
        out[2] = c;
    }
}

// ---------------------------------------------------------------------------
// The same op with the group term of the sparse-group penalty (Sec. III regulariser family):
//
//     u = prox_alpha(s - step g),   out_v = shrink u_v max(0, 1 - alpha_g / ||u_b||)
//
// over the 2 x 2 x 1 voxel blocks b = (ix/2, iy/2, iz) of an nx x ny x nz grid (x fastest; blocks at an
// odd edge hold fewer voxels).  One thread per block, its voxels in (dy, dx) order.
//
// Backward (o = shrink grad_out per voxel, real 2-vectors).  For ||u_b|| = n > alpha_g the block map
// u -> c u, c = 1 - alpha_g/n, has the symmetric Jacobian c I + (alpha_g/n^3) u u^T over the block, so
// grad_u = c o + (alpha_g/n^3) (sum_b o . u) u; d out/d alpha_g = -shrink u/n; d out/d shrink = c u.  For
// n <= alpha_g the block's output is 0 and nothing flows back.  grad_u then goes through the soft
// threshold as in prox_step_backward_kernel.
// ---------------------------------------------------------------------------
struct BlockIdx {
    long long v[4];     // voxel indices (x-fastest), valid for the first nv
    int nv;
};

__device__ __forceinline__ BlockIdx group_block(long long b, int nx, int ny, int gx, int gy)
{
    const long long per_plane = (long long)gx * gy;
    const int iz = (int)(b / per_plane);
    const long long r = b - iz * per_plane;
    const int by = (int)(r / gx), bx = (int)(r - (long long)by * gx);
    BlockIdx q;
    q.nv = 0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const int ix = 2 * bx + dx, iy = 2 * by + dy;
            if (ix < nx && iy < ny) q.v[q.nv++] = ((long long)iz * ny + iy) * nx + ix;
        }
    return q;
}

__global__ void prox_group_step_kernel(const float2* s, const float2* g, float step, float alpha, float alpha_g,
                                       float shrink, int nx, int ny, int nz, float2* out)
{
    const int gx = (nx + 1) / 2, gy = (ny + 1) / 2;
    const long long nb = (long long)gx * gy * nz;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
        const BlockIdx q = group_block(b, nx, ny, gx, gy);
        float2 u[4];
        float n2 = 0.f;
        for (int i = 0; i < q.nv; ++i) {
            u[i] = prox_one(s[q.v[i]], g[q.v[i]], step, alpha, 1.0f);
            n2 = fmaf(u[i].x, u[i].x, fmaf(u[i].y, u[i].y, n2));
        }
        const float nrm = sqrtf(n2);
        const float c = nrm > alpha_g ? (1.0f - alpha_g / nrm) * shrink : 0.f;
        for (int i = 0; i < q.nv; ++i) out[q.v[i]] = make_float2(c * u[i].x, c * u[i].y);
    }
}

// FP64 block partials [4 per CTA]: d/dstep, d/dalpha, d/dalpha_g, d/dshrink
__global__ void __launch_bounds__(256) prox_group_step_backward_kernel(const float2* s, const float2* g, float step,
                                                                       float alpha, float alpha_g, float shrink,
                                                                       int nx, int ny, int nz, const float2* go,
                                                                       float2* grad_s, float2* grad_g,
                                                                       double* partial)
{
    __shared__ double sh[4][256];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int gx = (nx + 1) / 2, gy = (ny + 1) / 2;
    const long long nb = (long long)gx * gy * nz;
    for (long long b = blockIdx.x * 256LL + threadIdx.x; b < nb; b += (long long)gridDim.x * 256) {
        const BlockIdx q = group_block(b, nx, ny, gx, gy);
        float2 z[4], u[4], o[4];
        float mag[4];
        float n2 = 0.f;
        for (int i = 0; i < q.nv; ++i) {
            const float2 sv = s[q.v[i]], gv = g[q.v[i]], o0 = go[q.v[i]];
            z[i] = make_float2(fmaf(-step, gv.x, sv.x), fmaf(-step, gv.y, sv.y));
            mag[i] = sqrtf(z[i].x * z[i].x + z[i].y * z[i].y);
            const float sc = mag[i] > alpha ? 1.0f - alpha / mag[i] : 0.f;
            u[i] = make_float2(z[i].x * sc, z[i].y * sc);
            o[i] = make_float2(shrink * o0.x, shrink * o0.y);
            n2 = fmaf(u[i].x, u[i].x, fmaf(u[i].y, u[i].y, n2));
        }
        const float nrm = sqrtf(n2);
        const bool live = nrm > alpha_g;
        float S = 0.f;                              // sum over the block of o . u
        for (int i = 0; i < q.nv; ++i) S = fmaf(o[i].x, u[i].x, fmaf(o[i].y, u[i].y, S));
        const float c = live ? 1.0f - alpha_g / nrm : 0.f;
        const float kb = live ? alpha_g / (nrm * nrm * nrm) * S : 0.f;
        if (live) {
            acc[2] -= (double)S / (double)nrm;
            acc[3] += (double)c * (double)S / (double)shrink;    // sum grad_out . (c u)
        }
        for (int i = 0; i < q.nv; ++i) {
            const float2 gu = make_float2(fmaf(c, o[i].x, kb * u[i].x), fmaf(c, o[i].y, kb * u[i].y));
            float2 gz = make_float2(0.f, 0.f);
            if (mag[i] > alpha) {
                const float sc = 1.0f - alpha / mag[i];
                const float zo = z[i].x * gu.x + z[i].y * gu.y;
                const float k = alpha / (mag[i] * mag[i] * mag[i]) * zo;
                gz = make_float2(fmaf(sc, gu.x, k * z[i].x), fmaf(sc, gu.y, k * z[i].y));
                acc[1] -= (double)zo / (double)mag[i];
            }
            const float2 gv = g[q.v[i]];
            if (grad_s) grad_s[q.v[i]] = gz;
            if (grad_g) grad_g[q.v[i]] = make_float2(-step * gz.x, -step * gz.y);
            acc[0] -= (double)gz.x * gv.x + (double)gz.y * gv.y;
        }
    }
    for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void sum_quads_kernel(const double* partial, int nb, double* out)
{
    if (threadIdx.x < 4 && blockIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < nb; ++i) a += partial[4 * i + threadIdx.x];
        out[threadIdx.x] = a;
    }
}

cudaError_t launch_prox_group_step(const float2* s, const float2* g, float step, float alpha, float alpha_g,
                                   float shrink, int nx, int ny, int nz, float2* out, cudaStream_t st)
{
    const long long nb = (long long)((nx + 1) / 2) * ((ny + 1) / 2) * nz;
    long long blocks = (nb + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    prox_group_step_kernel<<<(int)blocks, 256, 0, st>>>(s, g, step, alpha, alpha_g, shrink, nx, ny, nz, out);
    return cudaGetLastError();
}

cudaError_t launch_prox_group_step_backward(const float2* s, const float2* g, float step, float alpha, float alpha_g,
                                            float shrink, int nx, int ny, int nz, const float2* go, float2* grad_s,
                                            float2* grad_g, double* partial, double* out4, cudaStream_t st)
{
    prox_group_step_backward_kernel<<<RED_BLOCKS, 256, 0, st>>>(s, g, step, alpha, alpha_g, shrink, nx, ny, nz, go,
                                                                grad_s, grad_g, partial);
    sum_quads_kernel<<<1, 32, 0, st>>>(partial, RED_BLOCKS, out4);
    return cudaGetLastError();
}

cudaError_t launch_prox_step(const float2* s, const float2* g, float step, float alpha, float shrink, long long n,
                             float2* out, cudaStream_t st)
{
    const bool vec = ((uintptr_t)s % 16 == 0) && ((uintptr_t)g % 16 == 0) && ((uintptr_t)out % 16 == 0);
    if (vec && n >= 2) {
        const long long n2 = n / 2;
        long long blocks = (n2 + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        prox_step_vec_kernel<<<(int)blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(s),
                                                          reinterpret_cast<const float4*>(g), step, alpha, shrink,
                                                          n2, reinterpret_cast<float4*>(out));
        if (n % 2) prox_step_kernel<<<1, 32, 0, st>>>(s + n - 1, g + n - 1, step, alpha, shrink, 1, out + n - 1);
        return cudaGetLastError();
    }
    long long blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    prox_step_kernel<<<(int)blocks, 256, 0, st>>>(s, g, step, alpha, shrink, n, out);
    return cudaGetLastError();
}

cudaError_t launch_prox_step_backward(const float2* s, const float2* g, float step, float alpha, float shrink,
                                      long long n, const float2* go, float2* grad_s, float2* grad_g, double* partial,
                                      double* out3, cudaStream_t st)
{
    prox_step_backward_kernel<<<RED_BLOCKS, 256, 0, st>>>(s, g, step, alpha, shrink, n, go, grad_s, grad_g, partial);
    sum_triples_kernel<<<1, 32, 0, st>>>(partial, RED_BLOCKS, out3);
    return cudaGetLastError();
}

}  // namespace nfm
