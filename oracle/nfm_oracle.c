/*
 * Plain FP64 CPU oracle for the near-field MIMO observation operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or run this code.  It shares no code,
 * header or constant with the CUDA library.
 *
 * What it computes (Sec. II, Eq. 2):
 *   A[m][n] = p(f_m) * exp(-j 2 pi f_m (|r_Tm - r_n| + |r_Rm - r_n|) / c)
 *             / (4 pi |r_Tm - r_n| |r_Rm - r_n|)
 * with row m = pair * K + k, pair = t * R + r (TX index t, RX index r,
 * frequency index k) and voxel n = (iz * ny + iy) * nx + ix on a regular grid
 * r_n = (x0 + ix dx, y0 + iy dy, z0 + iz dz), or voxel n at the explicit
 * position pos[3n .. 3n + 2] when a point list is given.
 *
 * Every element is evaluated directly from the formula: two FP64 distances, the
 * phase f (dT + dR) / c in cycles with its nearest integer removed (exp of
 * -j 2 pi x is periodic in x with period 1, so this only removes whole turns
 * before cos/sin), and libm cos/sin.  No recurrence, no separability, no
 * tiling.  Sums run sequentially in index order; OpenMP splits only the
 * independent outputs (rows of the forward, columns of the adjoint), so the
 * result does not depend on the thread count.
 */
#include <math.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int T, R, K;
    const double* tx;     /* [T][3] */
    const double* rx;     /* [R][3] */
    const double* freq;   /* [K] Hz */
    const double* pulse;  /* [K][2] complex p(f_k), or NULL for p = 1 */
    double x0, y0, z0, dx, dy, dz;
    long nx, ny, nz;
    double c;
    const double* pos;    /* [N][3] explicit voxel positions, or NULL for the grid */
} orc_geom;

static const double ORC_PI = 3.14159265358979323846;

static void voxel_position(const orc_geom* g, long n, double* px, double* py, double* pz)
{
    if (g->pos) {
        *px = g->pos[3 * n];
        *py = g->pos[3 * n + 1];
        *pz = g->pos[3 * n + 2];
        return;
    }
    long ix = n % g->nx;
    long iy = (n / g->nx) % g->ny;
    long iz = n / (g->nx * g->ny);
    *px = g->x0 + (double)ix * g->dx;
    *py = g->y0 + (double)iy * g->dy;
    *pz = g->z0 + (double)iz * g->dz;
}

static double distance(const double* a, double x, double y, double z)
{
    double ex = a[0] - x, ey = a[1] - y, ez = a[2] - z;
    return sqrt(ex * ex + ey * ey + ez * ez);
}

/* A[m][n] of Eq. 2 -> out[0] (real), out[1] (imag). */
void orc_element(const orc_geom* g, long m, long n, double* out)
{
    long pair = m / g->K;
    int k = (int)(m % g->K);
    int t = (int)(pair / g->R);
    int r = (int)(pair % g->R);
    double x, y, z;
    voxel_position(g, n, &x, &y, &z);
    double dT = distance(g->tx + 3 * t, x, y, z);
    double dR = distance(g->rx + 3 * r, x, y, z);
    double cycles = g->freq[k] * (dT + dR) / g->c;
    cycles -= nearbyint(cycles);
    double amp = 1.0 / (4.0 * ORC_PI * dT * dR);
    double re = amp * cos(2.0 * ORC_PI * cycles);
    double im = -amp * sin(2.0 * ORC_PI * cycles);
    if (g->pulse) {
        double pr = g->pulse[2 * k], pi = g->pulse[2 * k + 1];
        double tr = pr * re - pi * im;
        double ti = pr * im + pi * re;
        re = tr;
        im = ti;
    }
    out[0] = re;
    out[1] = im;
}

/* Dense block A[rows][cols] -> out[nrows][ncols][2]. */
void orc_dense(const orc_geom* g, const long* rows, long nrows, const long* cols, long ncols, double* out)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nrows; ++i)
        for (long j = 0; j < ncols; ++j)
            orc_element(g, rows[i], cols[j], out + 2 * (i * ncols + j));
}

/* y[i] = sum_j A[rows[i]][cols[j]] * s[j]   (complex, interleaved). */
void orc_forward(const orc_geom* g, const long* rows, long nrows, const long* cols, long ncols,
                 const double* s, double* y)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < nrows; ++i) {
        double acc_re = 0.0, acc_im = 0.0, a[2];
        for (long j = 0; j < ncols; ++j) {
            orc_element(g, rows[i], cols[j], a);
            double sr = s[2 * j], si = s[2 * j + 1];
            acc_re += a[0] * sr - a[1] * si;
            acc_im += a[0] * si + a[1] * sr;
        }
        y[2 * i] = acc_re;
        y[2 * i + 1] = acc_im;
    }
}

/* out[j] = sum_i conj(A[rows[i]][cols[j]]) * r[i]   (the adjoint A^H r). */
void orc_adjoint(const orc_geom* g, const long* rows, long nrows, const double* r,
                 const long* cols, long ncols, double* out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long j = 0; j < ncols; ++j) {
        double acc_re = 0.0, acc_im = 0.0, a[2];
        for (long i = 0; i < nrows; ++i) {
            orc_element(g, rows[i], cols[j], a);
            double rr = r[2 * i], ri = r[2 * i + 1];
            /* conj(a) * r = (a0 - j a1)(rr + j ri) */
            acc_re += a[0] * rr + a[1] * ri;
            acc_im += a[0] * ri - a[1] * rr;
        }
        out[2 * j] = acc_re;
        out[2 * j + 1] = acc_im;
    }
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
