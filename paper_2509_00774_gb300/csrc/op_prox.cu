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
