// Set-up and reduction kernels: the FP64 per-(antenna, tile) tables and the
// FP64 norms / sums used by the power iteration, the objective (Eq. 3-4) and
// lambda_max.  Reductions use a fixed grid and a fixed tree, so their results
// do not depend on scheduling.
#include "nfm_kernels.cuh"

namespace nfm {

// For antenna a and tile t (centre r_c): v = r_a - r_c, |v|, and the phases
// f0|v|/c, df|v|/c, K2 df|v|/c reduced to [-1/2, 1/2] turns, all in FP64
// before the final rounding to FP32 (hi + lo for the two steps).
__global__ void ant_setup_kernel(GridDesc g, AntSetup a)
{
    const long long total = (long long)a.n_ant * g.n_tiles;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int ant = (int)(i / g.n_tiles);
        int tile = (int)(i - (long long)ant * g.n_tiles);
        double cx, cy, cz;
        if (a.tile_c) {                      // explicit voxel positions: the tile's own centre
            cx = a.tile_c[3 * (size_t)tile];
            cy = a.tile_c[3 * (size_t)tile + 1];
            cz = a.tile_c[3 * (size_t)tile + 2];
        } else {
            int tx, ty, tz;
            tile_coords(g, tile, tx, ty, tz);
            cx = a.x0 + (tx * TILE_X + 0.5 * (TILE_X - 1)) * a.dx;
            cy = a.y0 + (ty * TILE_Y + 0.5 * (TILE_Y - 1)) * a.dy;
            cz = a.z0 + (tz * TILE_Z + 0.5 * (TILE_Z - 1)) * a.dz;
        }
        double vx = a.ant_xyz[3 * ant + 0] - cx;
        double vy = a.ant_xyz[3 * ant + 1] - cy;
        double vz = a.ant_xyz[3 * ant + 2] - cz;
        double d2 = vx * vx + vy * vy + vz * vz;
        double d = sqrt(d2);
        double b = a.f0c * d;
        b -= rint(b);
        double s = a.dfc * d;
        s -= rint(s);
        double s2 = a.dfc2 * d;
        s2 -= rint(s2);
        AntTile o;
        o.vx = (float)vx;
        o.vy = (float)vy;
        o.vz = (float)vz;
        o.dc = (float)d;
        o.dc2 = (float)d2;
        o.b = (float)b;
        o.s_hi = (float)s;
        o.s_lo = (float)(s - (double)o.s_hi);
        o.s2_hi = (float)s2;
        o.s2_lo = (float)(s2 - (double)o.s2_hi);
        o.pad0 = 0.f;
        o.pad1 = 0.f;
        a.out[i] = o;
    }
}

cudaError_t launch_ant_setup(const GridDesc& g, const AntSetup& a, cudaStream_t st)
{
    long long total = (long long)a.n_ant * g.n_tiles;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    ant_setup_kernel<<<blocks, 256, 0, st>>>(g, a);
    return cudaGetLastError();
}

enum RedOp { RED_NORM2 = 0, RED_ABS_SUM = 1, RED_ABS_MAX = 2 };

template <int OP>
__device__ __forceinline__ double red_elem(float2 v)
{
    double x = v.x, y = v.y;
    if (OP == RED_NORM2) return x * x + y * y;
    return sqrt(x * x + y * y);
}

template <int OP>
__device__ __forceinline__ double red_comb(double a, double b)
{
    if (OP == RED_ABS_MAX) return a > b ? a : b;
    return a + b;
}

template <int OP>
__global__ void __launch_bounds__(256) reduce_partial_kernel(const float2* v, long long n, double* partial)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        acc = red_comb<OP>(acc, red_elem<OP>(v[i]));
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = red_comb<OP>(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

template <int OP>
__global__ void __launch_bounds__(256) reduce_final_kernel(const double* partial, int n, double* out)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) acc = red_comb<OP>(acc, partial[i]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = red_comb<OP>(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

template <int OP>
static cudaError_t launch_reduce(const float2* v, long long n, double* partial, double* out, cudaStream_t st)
{
    reduce_partial_kernel<OP><<<RED_BLOCKS, 256, 0, st>>>(v, n, partial);
    reduce_final_kernel<OP><<<1, 256, 0, st>>>(partial, RED_BLOCKS, out);
    return cudaGetLastError();
}

cudaError_t launch_norm2(const float2* v, long long n, double* partial, double* out, cudaStream_t st)
{
    return launch_reduce<RED_NORM2>(v, n, partial, out, st);
}

cudaError_t launch_abs_sum(const float2* v, long long n, double* partial, double* out, cudaStream_t st)
{
    return launch_reduce<RED_ABS_SUM>(v, n, partial, out, st);
}

cudaError_t launch_abs_max(const float2* v, long long n, double* partial, double* out, cudaStream_t st)
{
    return launch_reduce<RED_ABS_MAX>(v, n, partial, out, st);
}

__global__ void __launch_bounds__(256) group_norm_partial_kernel(const float2* v, int nx, int ny, int nz,
                                                                 double* partial)
{
    __shared__ double sh[256];
    const int gx = (nx + 1) / 2, gy = (ny + 1) / 2;
    const long long n_groups = (long long)gx * gy * nz;
    double acc = 0.0;
    for (long long g = blockIdx.x * 256LL + threadIdx.x; g < n_groups; g += (long long)gridDim.x * 256) {
        const int bx = (int)(g % gx);
        const long long rest = g / gx;
        const int by = (int)(rest % gy), iz = (int)(rest / gy);
        double s2 = 0.0;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int ix = 2 * bx + dx, iy = 2 * by + dy;
                if (ix < nx && iy < ny) {
                    const float2 x = v[((size_t)iz * ny + iy) * nx + ix];
                    s2 += (double)x.x * x.x + (double)x.y * x.y;
                }
            }
        acc += sqrt(s2);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

cudaError_t launch_group_norm_sum(const float2* v, int nx, int ny, int nz, double* partial, double* out,
                                  cudaStream_t st)
{
    group_norm_partial_kernel<<<RED_BLOCKS, 256, 0, st>>>(v, nx, ny, nz, partial);
    reduce_final_kernel<RED_ABS_SUM><<<1, 256, 0, st>>>(partial, RED_BLOCKS, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) mag_change_partial_kernel(const float2* a, const float2* b, long long n,
                                                                 double* partial)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float2 x = a[i], y = b[i];
        const double d = fabs(sqrt((double)x.x * x.x + (double)x.y * x.y) - sqrt((double)y.x * y.x + (double)y.y * y.y));
        acc = d > acc ? d : acc;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

cudaError_t launch_mag_change(const float2* a, const float2* b, long long n, double* partial, double* out,
                              cudaStream_t st)
{
    mag_change_partial_kernel<<<RED_BLOCKS, 256, 0, st>>>(a, b, n, partial);
    reduce_final_kernel<RED_ABS_MAX><<<1, 256, 0, st>>>(partial, RED_BLOCKS, out);
    return cudaGetLastError();
}

__global__ void normalize_kernel(const float2* src, float2* dst, long long n, const double* nrm2)
{
    const double nv = nrm2[0];
    const float sc = nv > 0.0 ? (float)(1.0 / sqrt(nv)) : 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float2 x = src[i];
        dst[i] = make_float2(x.x * sc, x.y * sc);
    }
}

cudaError_t launch_normalize(const float2* src, float2* dst, long long n, const double* nrm2, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    normalize_kernel<<<(int)blocks, 256, 0, st>>>(src, dst, n, nrm2);
    return cudaGetLastError();
}

__global__ void ratio_kernel(const double* a, const double* b, double scale, double* out)
{
    out[0] = a[0] / (scale * b[0]);
}

cudaError_t launch_ratio(const double* a, const double* b, double scale, double* out, cudaStream_t st)
{
    ratio_kernel<<<1, 1, 0, st>>>(a, b, scale, out);
    return cudaGetLastError();
}

__global__ void axpby_kernel(const double* a, double sa, const double* b, double sb, double* out)
{
    out[0] = a[0] * sa + b[0] * sb;
}

cudaError_t launch_axpby(const double* a, double sa, const double* b, double sb, double* out, cudaStream_t st)
{
    axpby_kernel<<<1, 1, 0, st>>>(a, sa, b, sb, out);
    return cudaGetLastError();
}

}  // namespace nfm
