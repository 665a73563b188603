/*
 * FP64 reference ("oracle") for the sliding Frank-Wolfe hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header or constant with the CUDA
 * path.
 *
 * Every function is the plain definition, written out as nested loops over
 * voxels, in double precision, without truncation, blocking or reordering.
 * OpenMP only splits the outermost loop; each output is still the same
 * sequential sum.
 *
 * Geometry.  The observation grid has shape n = (n0, n1, n2), C-contiguous,
 * axis 2 fastest, voxel centres at integer coordinates 0..n_a-1.  The PSF H
 * has shape (2R0+1, 2R1+1, 2R2+1) and is centred at index R.  Atoms are
 * sampled on the extended grid E of shape n + 2R: E index t holds the point
 * of grid coordinate t - R.  With this reading the blurred observation of
 * Eq. 3, restricted to the grid, is an exact finite sum, and so is its
 * adjoint (the transposed operator of Eq. 5).
 *
 * Atom (Eq. 2): G(theta, w; s) = w exp(-(1/(2 sigma^d)) |m - s|^d),
 *               theta = (m, sigma, d).
 *
 * Parameter vector order for gradients (6 per atom, "6 = dim D" in
 * Section 2 read as (m, sigma, d) plus w):
 *   grad[3n + a]   = dC/dm_{n,a}      a = 0,1,2
 *   grad[3N + n]   = dC/dsigma_n
 *   grad[4N + n]   = dC/dd_n
 *   grad[5N + n]   = dC/dw_n
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX3(i, j, k, n1, n2) ((((size_t)(i)) * (size_t)(n1) + (size_t)(j)) * (size_t)(n2) + (size_t)(k))

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Generalised isotropic Gaussian of Eq. 2 with unit weight, at squared
 * distance rho2 from its centre: exp(-(1/2) (rho/sigma)^d). */
static double atom_profile(double rho2, double sigma, double d) {
    if (rho2 <= 0.0) return 1.0;
    double rho = sqrt(rho2);
    return exp(-0.5 * pow(rho / sigma, d));
}

/* Render f(t) = sum_n w_n exp(-(1/2)(|t - R - m_n| / sigma_n)^{d_n}) on E
 * (Eq. 2 summed over the atoms of mu, as inside Eq. 3). */
void oracle_render(const int n[3], const int R[3], int N, const double* m,
                   const double* sigma, const double* d, const double* w, double* f) {
    const int E0 = n[0] + 2 * R[0], E1 = n[1] + 2 * R[1], E2 = n[2] + 2 * R[2];
#pragma omp parallel for schedule(static)
    for (int t0 = 0; t0 < E0; ++t0) {
        for (int t1 = 0; t1 < E1; ++t1) {
            for (int t2 = 0; t2 < E2; ++t2) {
                double x0 = (double)(t0 - R[0]), x1 = (double)(t1 - R[1]), x2 = (double)(t2 - R[2]);
                double acc = 0.0;
                for (int a = 0; a < N; ++a) {
                    double e0 = x0 - m[3 * a + 0], e1 = x1 - m[3 * a + 1], e2 = x2 - m[3 * a + 2];
                    acc += w[a] * atom_profile(e0 * e0 + e1 * e1 + e2 * e2, sigma[a], d[a]);
                }
                f[IDX3(t0, t1, t2, E1, E2)] = acc;
            }
        }
    }
}

/* Blur and observe on the grid (Eq. 3): y(s) = sum_{t in E} H(s - t) f(t),
 * H(u) stored at index u + R.  Only t with |s + R - t|_a <= R_a contribute. */
void oracle_forward_conv(const int n[3], const int R[3], const double* psf, const double* f,
                         double* y) {
    const int E1 = n[1] + 2 * R[1], E2 = n[2] + 2 * R[2];
    const int H1 = 2 * R[1] + 1, H2 = 2 * R[2] + 1;
#pragma omp parallel for schedule(static)
    for (int s0 = 0; s0 < n[0]; ++s0) {
        for (int s1 = 0; s1 < n[1]; ++s1) {
            for (int s2 = 0; s2 < n[2]; ++s2) {
                double acc = 0.0;
                /* u = s - t in [-R, R]  <=>  t = s + R - (u + R), E index */
                for (int u0 = -R[0]; u0 <= R[0]; ++u0)
                    for (int u1 = -R[1]; u1 <= R[1]; ++u1)
                        for (int u2 = -R[2]; u2 <= R[2]; ++u2) {
                            int t0 = s0 + R[0] - u0, t1 = s1 + R[1] - u1, t2 = s2 + R[2] - u2;
                            acc += psf[IDX3(u0 + R[0], u1 + R[1], u2 + R[2], H1, H2)] *
                                   f[IDX3(t0, t1, t2, E1, E2)];
                        }
                y[IDX3(s0, s1, s2, n[1], n[2])] = acc;
            }
        }
    }
}

/* Adjoint of oracle_forward_conv (the Phi^T of Eq. 5 before sampling the atom):
 * b(t) = sum_{s in grid} H(s - t) r(s) for every t in E. */
void oracle_backproject(const int n[3], const int R[3], const double* psf, const double* r,
                        double* b) {
    const int E0 = n[0] + 2 * R[0], E1 = n[1] + 2 * R[1], E2 = n[2] + 2 * R[2];
    const int H1 = 2 * R[1] + 1, H2 = 2 * R[2] + 1;
#pragma omp parallel for schedule(static)
    for (int t0 = 0; t0 < E0; ++t0) {
        for (int t1 = 0; t1 < E1; ++t1) {
            for (int t2 = 0; t2 < E2; ++t2) {
                double acc = 0.0;
                /* u = s - (t - R) in [-R, R]; only s inside the grid observe */
                for (int u0 = -R[0]; u0 <= R[0]; ++u0) {
                    int s0 = t0 - R[0] + u0;
                    if (s0 < 0 || s0 >= n[0]) continue;
                    for (int u1 = -R[1]; u1 <= R[1]; ++u1) {
                        int s1 = t1 - R[1] + u1;
                        if (s1 < 0 || s1 >= n[1]) continue;
                        for (int u2 = -R[2]; u2 <= R[2]; ++u2) {
                            int s2 = t2 - R[2] + u2;
                            if (s2 < 0 || s2 >= n[2]) continue;
                            acc += psf[IDX3(u0 + R[0], u1 + R[1], u2 + R[2], H1, H2)] *
                                   r[IDX3(s0, s1, s2, n[1], n[2])];
                        }
                    }
                }
                b[IDX3(t0, t1, t2, E1, E2)] = acc;
            }
        }
    }
}

/* Certificate of Eq. 5 at arbitrary parameters:
 *   eta(theta) = (1/lambda) <Phi G(theta, 1), r> = (1/lambda) sum_{t in E} g_theta(t) b(t),
 * with b = Phi^T-backprojection of the residual on E (oracle_backproject).
 * theta is P x 5: (m0, m1, m2, sigma, d).  If grad != NULL it also returns
 * d eta / d theta (P x 5), used by the local ascent of step 1. */
void oracle_eta_points(const int n[3], const int R[3], const double* b, double lambda, int P,
                       const double* theta, double* eta, double* grad) {
    const int E0 = n[0] + 2 * R[0], E1 = n[1] + 2 * R[1], E2 = n[2] + 2 * R[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        const double m0 = theta[5 * p + 0], m1 = theta[5 * p + 1], m2 = theta[5 * p + 2];
        const double sg = theta[5 * p + 3], dd = theta[5 * p + 4];
        double acc = 0.0, gm0 = 0.0, gm1 = 0.0, gm2 = 0.0, gs = 0.0, gd = 0.0;
        for (int t0 = 0; t0 < E0; ++t0)
            for (int t1 = 0; t1 < E1; ++t1)
                for (int t2 = 0; t2 < E2; ++t2) {
                    double e0 = (double)(t0 - R[0]) - m0, e1 = (double)(t1 - R[1]) - m1,
                           e2 = (double)(t2 - R[2]) - m2;
                    double rho2 = e0 * e0 + e1 * e1 + e2 * e2;
                    double bt = b[IDX3(t0, t1, t2, E1, E2)];
                    if (rho2 <= 0.0) {
                        acc += bt; /* g = 1; dg/dm = dg/dsigma = dg/dd = 0 at rho = 0 */
                        continue;
                    }
                    double rho = sqrt(rho2);
                    double u = 0.5 * pow(rho / sg, dd);
                    double g = exp(-u);
                    acc += g * bt;
                    if (grad) {
                        /* dg/dm_a = -g d u (m_a - x_a)/rho^2 = +g d u e_a / rho^2 (e = x - m) */
                        double c = g * dd * u / rho2 * bt;
                        gm0 += c * e0;
                        gm1 += c * e1;
                        gm2 += c * e2;
                        gs += g * (dd / sg) * u * bt;
                        gd += -g * u * log(rho / sg) * bt;
                    }
                }
        eta[p] = acc / lambda;
        if (grad) {
            grad[5 * p + 0] = gm0 / lambda;
            grad[5 * p + 1] = gm1 / lambda;
            grad[5 * p + 2] = gm2 / lambda;
            grad[5 * p + 3] = gs / lambda;
            grad[5 * p + 4] = gd / lambda;
        }
    }
}

/* Analytic gradient of the criterion C of Eq. 4 with respect to all 6N atom
 * parameters, given b = backprojection of r = y - Phi mu on E:
 *   dC/dw_n     = lambda - sum_t g_n(t) b(t)
 *   dC/dtheta_n = -w_n sum_t (d g_n / d theta)(t) b(t)
 * with u = (1/2)(rho/sigma)^d, g = exp(-u):
 *   dg/dsigma = g (d/sigma) u,  dg/dd = -g u ln(rho/sigma),
 *   dg/dm_a   = -g d u (m_a - x_a) / rho^2, all three zero at rho = 0. */
void oracle_atom_grad(const int n[3], const int R[3], int N, const double* m, const double* sigma,
                      const double* d, const double* w, const double* b, double lambda,
                      double* grad) {
    const int E0 = n[0] + 2 * R[0], E1 = n[1] + 2 * R[1], E2 = n[2] + 2 * R[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < N; ++a) {
        const double sg = sigma[a], dd = d[a];
        double sg_b = 0.0, sm0 = 0.0, sm1 = 0.0, sm2 = 0.0, ss = 0.0, sd = 0.0;
        for (int t0 = 0; t0 < E0; ++t0)
            for (int t1 = 0; t1 < E1; ++t1)
                for (int t2 = 0; t2 < E2; ++t2) {
                    double x0 = (double)(t0 - R[0]), x1 = (double)(t1 - R[1]), x2 = (double)(t2 - R[2]);
                    double e0 = m[3 * a + 0] - x0, e1 = m[3 * a + 1] - x1, e2 = m[3 * a + 2] - x2;
                    double rho2 = e0 * e0 + e1 * e1 + e2 * e2;
                    double bt = b[IDX3(t0, t1, t2, E1, E2)];
                    if (rho2 <= 0.0) {
                        sg_b += bt;
                        continue;
                    }
                    double rho = sqrt(rho2);
                    double u = 0.5 * pow(rho / sg, dd);
                    double g = exp(-u);
                    sg_b += g * bt;
                    double c = -g * dd * u / rho2 * bt; /* (dg/dm_a) b = c (m_a - x_a) */
                    sm0 += c * e0;
                    sm1 += c * e1;
                    sm2 += c * e2;
                    ss += g * (dd / sg) * u * bt;
                    sd += -g * u * log(rho / sg) * bt;
                }
        grad[3 * a + 0] = -w[a] * sm0;
        grad[3 * a + 1] = -w[a] * sm1;
        grad[3 * a + 2] = -w[a] * sm2;
        grad[3 * N + a] = -w[a] * ss;
        grad[4 * N + a] = -w[a] * sd;
        grad[5 * N + a] = lambda - sg_b;
    }
}

/* Index of the largest value, ties to the lowest index; -1 if a NaN is present
 * (the certificate must be a real number everywhere). */
int64_t oracle_argmax(const double* v, int64_t count) {
    int64_t best = -1;
    for (int64_t i = 0; i < count; ++i) {
        if (v[i] != v[i]) return -1;
        if (best < 0 || v[i] > v[best]) best = i;
    }
    return best;
}
