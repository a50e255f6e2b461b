/*
 * FP64 oracle for the short-range particle-particle force.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a small host library
 * that the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load to check the CUDA path.  The library itself never calls it.
 *
 * What it computes is the plain definition, for every target particle i:
 *
 *   a_i = sum_{j != i, r_ij < rcut}  G m_j d_ij f(r_ij) / (r_ij^2 + eps^2)^{3/2}
 *
 *   d_ij = x_j - x_i - L round((x_j - x_i)/L)   per axis (minimum image,
 *                                                 periodic box)
 *   f(s) = erfc(s / 2R_s) + s/(R_s sqrt(pi)) exp(-s^2 / 4R_s^2)
 *
 * f is the short-range split factor of Eq. (split) (Sec. 3.1), applied to the
 * Newtonian pair force G m_j d/r^3 as in the PM-Tree scheme the paper follows;
 * the cutoff rcut is the R_cut of Sec. 3.1 beyond which the short-range force
 * is dropped; Plummer softening enters only the Newtonian factor, f is taken
 * at the unsoftened separation.  Every pair is summed directly, all sources
 * against each target, in double precision: no tree, no lists, no blocking.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (fp contraction off
 * so that x86 and Arm hosts give the same bits).
 */
#include <math.h>
#include <stdint.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Eq. (split): the short-range factor at separation s for split scale rs. */
double phor_split_factor(double s, double rs)
{
    double a = s / (2.0 * rs);
    return erfc(a) + s / (rs * sqrt(M_PI)) * exp(-(s * s) / (4.0 * rs * rs));
}

void phor_split_factor_v(int64_t n, const double *s, double rs, double *out)
{
    for (int64_t k = 0; k < n; k++) out[k] = phor_split_factor(s[k], rs);
}

static double min_image(double d, double L)
{
    return d - L * round(d / L);
}

/*
 * Acceleration of each target.
 *
 *   pos      [n*3]  source positions (any real coordinates; min image is
 *                   applied to differences)
 *   mass     [n]
 *   targets  [nt]   indices of the targets, or NULL for targets 0..nt-1
 *   acc      [nt*3] out: accelerations
 *   abs_sum  [nt]   out (nullable): sum over contributing j of |term_ij|
 *   n_within [nt]   out (nullable): number of j with r < rcut, j != i
 *   near_abs [nt]   out (nullable): sum of |term| over pairs whose separation
 *                   lies within near_tol*rcut of rcut (either side), i.e. the
 *                   pairs a single-precision cutoff test may classify either
 *                   way; the term is evaluated at the pair's r even if r >= rcut
 */
void phor_accel(int64_t n, const double *pos, const double *mass,
                double L, double G, double eps, double rs, double rcut,
                int64_t nt, const int64_t *targets,
                double *acc, double *abs_sum, int64_t *n_within,
                double *near_abs, double near_tol)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < nt; t++) {
        const int64_t i = targets ? targets[t] : t;
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        double ax = 0.0, ay = 0.0, az = 0.0, sabs = 0.0, snear = 0.0;
        int64_t cnt = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = min_image(pos[3 * j] - xi, L);
            double dy = min_image(pos[3 * j + 1] - yi, L);
            double dz = min_image(pos[3 * j + 2] - zi, L);
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            int near = fabs(r - rcut) <= near_tol * rcut;
            if (!(r < rcut) && !near) continue;
            double re2 = r2 + eps2;
            double w = G * mass[j] * phor_split_factor(r, rs) / (re2 * sqrt(re2));
            if (near) snear += fabs(w) * r;
            if (!(r < rcut)) continue;
            ax += w * dx;
            ay += w * dy;
            az += w * dz;
            sabs += fabs(w) * r;
            cnt++;
        }
        acc[3 * t] = ax;
        acc[3 * t + 1] = ay;
        acc[3 * t + 2] = az;
        if (abs_sum) abs_sum[t] = sabs;
        if (n_within) n_within[t] = cnt;
        if (near_abs) near_abs[t] = snear;
    }
}

/*
 * The learned factor: the 1-16-16-1 SiLU network evaluated in double at
 * z0 = 2 r / rcut - 1.  w[321] = W1[16], b1[16], W2[16][16] (row k = weights
 * into unit k), b2[16], W3[16], b3.
 */
static double silu(double a) { return a / (1.0 + exp(-a)); }

double phor_mlp_factor(const double *w, double r, double rcut)
{
    const double *W1 = w, *b1 = w + 16, *W2 = w + 32, *b2 = w + 288, *W3 = w + 304, b3 = w[320];
    double z0 = 2.0 * r / rcut - 1.0, h1[16], y = b3;
    for (int j = 0; j < 16; j++) h1[j] = silu(W1[j] * z0 + b1[j]);
    for (int k = 0; k < 16; k++) {
        double a = b2[k];
        for (int j = 0; j < 16; j++) a += W2[16 * k + j] * h1[j];
        y += W3[k] * silu(a);
    }
    return y;
}

/* Same sum as phor_accel with the network standing in for Eq. (split). */
void phor_accel_mlp(int64_t n, const double *pos, const double *mass, double L, double G, double eps,
                    double rcut, const double *w, int64_t nt, const int64_t *targets, double *acc)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < nt; t++) {
        const int64_t i = targets ? targets[t] : t;
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = min_image(pos[3 * j] - pos[3 * i], L);
            double dy = min_image(pos[3 * j + 1] - pos[3 * i + 1], L);
            double dz = min_image(pos[3 * j + 2] - pos[3 * i + 2], L);
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            if (!(r < rcut)) continue;
            double re2 = r2 + eps2;
            double wgt = G * mass[j] * phor_mlp_factor(w, r, rcut) / (re2 * sqrt(re2));
            ax += wgt * dx;
            ay += wgt * dy;
            az += wgt * dz;
        }
        acc[3 * t] = ax;
        acc[3 * t + 1] = ay;
        acc[3 * t + 2] = az;
    }
}

/* Number of threads OpenMP will use for the parallel loop above. */
int phor_num_threads(void)
{
    int nt = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            nt = omp_get_num_threads();
#endif
        }
    }
    return nt;
}
