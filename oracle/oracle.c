/*
 * FP64 CPU oracle for the Stokeslet + stresslet treecode
 * (Wang, Tlupova, Krasny, "A treecode algorithm for 3D Stokeslets and
 * stresslets", arXiv:1811.12498).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library; the two meet only at the seeded input generators.
 *
 * The oracle is deliberately plain and slow:
 *   - the direct sum is the definition of eq. (1.3) ("StoStre") with the
 *     kernel tensors S_ij and T_ijl of eqs. (1.2a,b) formed explicitly;
 *   - the treecode decides, target by target, which clusters are taken in
 *     the far field and which leaves are summed directly (the MAC of
 *     eq. 5.1 over the octree of Section 5, Algorithm 1's decisions), by an
 *     explicit-stack walk that records an interaction list, and then sums
 *     that list: cluster moments of Section 2 from their definition, the
 *     Coulomb coefficients from recurrence (3.2), the far field from the
 *     contracted forms (4.4) ("S_final") and (4.9) ("T_final"), the leaves
 *     by the contracted direct sum of Section 4.1;
 *   - the explicit Taylor coefficients a^k_ij (3.4) and a~^k_ijl (3.7) are
 *     provided as a cross-check of the contracted forms.
 * Multi-indices are held in plain (P+1)^3 cubes, zero outside ||k|| <= P.
 *
 * Readings of points the paper leaves open:
 *   - kernel prefactor 1 (Section 1 defines the kernels up to a constant);
 *   - a pair contributes nothing when |x - y| == 0 exactly (this is the
 *     n != m exclusion of eq. (1.3) when targets are the sources);
 *   - root cell: per-axis minimum corner, side = largest axis extent; cell
 *     membership follows 21-bit quantised coordinates, so a point on a
 *     bisection plane belongs to the upper child and the maximum point is
 *     clamped into the last cell (Section 5);
 *   - a cluster is a leaf iff it holds at most N0 particles or is at depth 21
 *     (Section 5 stops splitting below N0 particles, Section 6 treats N0 as
 *     the maximum leaf size);
 *   - cluster centre: centre of the tight bounding box (shrink = 1, test
 *     case 1) or centre of the octree cell (shrink = 0); radius r = max
 *     distance from the centre to the cluster's particles (Section 2);
 *   - MAC r/R <= theta (eq. 5.1) evaluated as R^2 > 0 and r^2 <= theta^2 R^2;
 *   - children are visited in octant order (x bit most significant).
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -shared -fPIC.
 * -ffp-contract=off matters: the quantisation, cell centres, radii and MAC
 * must round exactly as written so that tree decisions are reproducible.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXDEPTH 21
#define ORC_PMAX 12

/* ------------------------------------------------------------------ */
/* Kernels, eqs. (1.2a) and (1.2b).                                   */
/* ------------------------------------------------------------------ */

/* S_ij(x,y) = delta_ij/|x-y| + (x_i-y_i)(x_j-y_j)/|x-y|^3, row-major 3x3. */
void orc_stokeslet(const double* x, const double* y, double* S)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            S[3 * i + j] = (i == j ? 1.0 / r : 0.0) + d[i] * d[j] / (r * r * r);
}

/* T_ijl(x,y) = (x_i-y_i)(x_j-y_j)(x_l-y_l)/|x-y|^5, index 9i+3j+l. */
void orc_stresslet(const double* x, const double* y, double* T)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double r5 = r * r * r * r * r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                T[9 * i + 3 * j + l] = d[i] * d[j] * d[l] / r5;
}

/* ------------------------------------------------------------------ */
/* Direct sum, eq. (1.3), written from the definition.                 */
/* Arrays are row-major (count, 3).  Pairs with |x-y| == 0 are skipped.*/
/* ------------------------------------------------------------------ */
void orc_direct(const double* x, const double* f, const double* h, const double* nu,
                int64_t N, const double* tx, int64_t M, double* u, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; m++) {
        const double* xm = tx + 3 * m;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t n = 0; n < N; n++) {
            const double* yn = x + 3 * n;
            if (xm[0] == yn[0] && xm[1] == yn[1] && xm[2] == yn[2]) continue;
            double S[9], T[27];
            orc_stokeslet(xm, yn, S);
            orc_stresslet(xm, yn, T);
            for (int i = 0; i < 3; i++) {
                double s = 0.0;
                for (int j = 0; j < 3; j++) {
                    s += S[3 * i + j] * f[3 * n + j];
                    for (int l = 0; l < 3; l++)
                        s += T[9 * i + 3 * j + l] * h[3 * n + j] * nu[3 * n + l];
                }
                acc[i] += s;
            }
        }
        u[3 * m + 0] = acc[0];
        u[3 * m + 1] = acc[1];
        u[3 * m + 2] = acc[2];
    }
}

/* Gradient of L = sum_m g_m . u_m, u the direct sum of eq. (1.3) (targets
 * = sources, coincident pairs skipped), by differentiating S and T of
 * eqs. (1.2a,b) as defined: with d = x_m - x_n, r = |d|,
 *   dS_ij/dd_a = -delta_ij d_a / r^3 + (delta_ia d_j + d_i delta_ja) / r^3
 *                - 3 d_i d_j d_a / r^5,
 *   dT_ijl/dd_a = (delta_ia d_j d_l + d_i delta_ja d_l + d_i d_j delta_la) / r^5
 *                 - 5 d_i d_j d_l d_a / r^7;
 * dL/df_n = sum_m S(d)^T g_m, dL/dh_n,j = sum_m g_m,i T_ijl nu_n,l,
 * dL/dnu_n,l = sum_m g_m,i T_ijl h_n,j, and dL/dx gets +dphi/dd at the
 * target and -dphi/dd at the source of every pair.  Arrays are N x 3. */
static void pair_dphi(const double* d, const double* g, const double* f, const double* h, const double* nu,
                      double* out)
{
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
    for (int a = 0; a < 3; a++) {
        double s = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double dS = -((i == j) ? d[a] / r3 : 0.0) + (((i == a) ? d[j] : 0.0) + ((j == a) ? d[i] : 0.0)) / r3 -
                            3.0 * d[i] * d[j] * d[a] / r5;
                s += g[i] * dS * f[j];
                for (int l = 0; l < 3; l++) {
                    double dT = (((i == a) ? d[j] * d[l] : 0.0) + ((j == a) ? d[i] * d[l] : 0.0) +
                                 ((l == a) ? d[i] * d[j] : 0.0)) / r5 -
                                5.0 * d[i] * d[j] * d[l] * d[a] / r7;
                    s += g[i] * dT * h[j] * nu[l];
                }
            }
        out[a] = s;
    }
}

void orc_direct_grad(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                     const double* g, double* gf, double* gh, double* gnu, double* gx, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    /* source side: the weights of n and the source part of dL/dx_n */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t n = 0; n < N; n++) {
        const double* yn = x + 3 * n;
        double af[3] = {0, 0, 0}, ah[3] = {0, 0, 0}, an[3] = {0, 0, 0}, ax[3] = {0, 0, 0};
        for (int64_t m = 0; m < N; m++) {
            const double* xm = x + 3 * m;
            if (xm[0] == yn[0] && xm[1] == yn[1] && xm[2] == yn[2]) continue;
            double S[9], T[27], d[3] = {xm[0] - yn[0], xm[1] - yn[1], xm[2] - yn[2]}, dp[3];
            orc_stokeslet(xm, yn, S);
            orc_stresslet(xm, yn, T);
            const double* gm = g + 3 * m;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    af[j] += gm[i] * S[3 * i + j];
                    for (int l = 0; l < 3; l++) {
                        ah[j] += gm[i] * T[9 * i + 3 * j + l] * nu[3 * n + l];
                        an[l] += gm[i] * T[9 * i + 3 * j + l] * h[3 * n + j];
                    }
                }
            pair_dphi(d, gm, f + 3 * n, h + 3 * n, nu + 3 * n, dp);
            for (int a = 0; a < 3; a++) ax[a] -= dp[a];
        }
        for (int a = 0; a < 3; a++) {
            gf[3 * n + a] = af[a];
            gh[3 * n + a] = ah[a];
            gnu[3 * n + a] = an[a];
            gx[3 * n + a] = ax[a];
        }
    }
    /* target side: the target part of dL/dx_m */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < N; m++) {
        const double* xm = x + 3 * m;
        double ax[3] = {0, 0, 0};
        for (int64_t n = 0; n < N; n++) {
            const double* yn = x + 3 * n;
            if (xm[0] == yn[0] && xm[1] == yn[1] && xm[2] == yn[2]) continue;
            double d[3] = {xm[0] - yn[0], xm[1] - yn[1], xm[2] - yn[2]}, dp[3];
            pair_dphi(d, g + 3 * m, f + 3 * n, h + 3 * n, nu + 3 * n, dp);
            for (int a = 0; a < 3; a++) ax[a] += dp[a];
        }
        for (int a = 0; a < 3; a++) gx[3 * m + a] += ax[a];
    }
}

/* ------------------------------------------------------------------ */
/* Regularized kernels.  The paper closes by naming regularized        */
/* Stokeslets and stresslets as future work and gives neither kernel;  */
/* these follow the blob of Cortez, Fauci and Medovikov (Phys. Fluids  */
/* 17, 031504, 2005), phi(r) = 15 eps^4 / (8 pi (r^2 + eps^2)^(7/2)).  */
/* With s = r^2 + eps^2 and the normalisation of eqs. (1.2a,b):        */
/*   S^eps_ij = delta_ij (r^2 + 2 eps^2) / s^(3/2) + d_i d_j / s^(3/2), */
/* the velocity of a regularized point force, and                      */
/*   T^eps_ijl = [d_i d_j d_l + (eps^2/2)(delta_ij d_l + delta_jl d_i  */
/*               + delta_il d_j)] / s^(5/2),                           */
/* minus one sixth of that flow's stress, as T_ijl is of the singular  */
/* Stokeslet's.  At eps = 0 they are eqs. (1.2a,b).                    */
/* ------------------------------------------------------------------ */
void orc_stokeslet_reg(const double* x, const double* y, double eps, double* S)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double e2 = eps * eps, s = r2 + e2, s32 = s * sqrt(s);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) S[3 * i + j] = ((i == j ? r2 + 2.0 * e2 : 0.0) + d[i] * d[j]) / s32;
}

void orc_stresslet_reg(const double* x, const double* y, double eps, double* T)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double e2 = eps * eps, s = r2 + e2, s52 = s * s * sqrt(s);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++) {
                double v = d[i] * d[j] * d[l];
                v += 0.5 * e2 * ((i == j ? d[l] : 0.0) + (j == l ? d[i] : 0.0) + (i == l ? d[j] : 0.0));
                T[9 * i + 3 * j + l] = v / s52;
            }
}

/* eq. (1.3) with the regularized kernels; pairs with |x - y| == 0 are
 * skipped as in orc_direct (the n != m exclusion). */
void orc_direct_reg(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                    const double* tx, int64_t M, double eps, double* u, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; m++) {
        const double* xm = tx + 3 * m;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t n = 0; n < N; n++) {
            const double* yn = x + 3 * n;
            if (xm[0] == yn[0] && xm[1] == yn[1] && xm[2] == yn[2]) continue;
            double S[9], T[27];
            orc_stokeslet_reg(xm, yn, eps, S);
            orc_stresslet_reg(xm, yn, eps, T);
            for (int i = 0; i < 3; i++) {
                double sum = 0.0;
                for (int j = 0; j < 3; j++) {
                    sum += S[3 * i + j] * f[3 * n + j];
                    for (int l = 0; l < 3; l++) sum += T[9 * i + 3 * j + l] * h[3 * n + j] * nu[3 * n + l];
                }
                acc[i] += sum;
            }
        }
        u[3 * m + 0] = acc[0];
        u[3 * m + 1] = acc[1];
        u[3 * m + 2] = acc[2];
    }
}

/* ------------------------------------------------------------------ */
/* Multi-index cube helpers.  A cube of order P holds entries          */
/* (k1,k2,k3) with 0 <= k_a <= P; only ||k|| <= P are meaningful.      */
/* ------------------------------------------------------------------ */
static inline int cube_idx(int P, int k1, int k2, int k3)
{
    return (k1 * (P + 1) + k2) * (P + 1) + k3;
}

/* value of cube c at k, or 0 if any component is negative or ||k|| > P */
static inline double cube_at(const double* c, int P, int k1, int k2, int k3)
{
    if (k1 < 0 || k2 < 0 || k3 < 0) return 0.0;
    if (k1 + k2 + k3 > P) return 0.0;
    return c[cube_idx(P, k1, k2, k3)];
}

/* ------------------------------------------------------------------ */
/* Coulomb Taylor coefficients b^k(x, y_c), ||k|| <= P, recurrence     */
/* (3.2): ||k|| R^2 b^k - (2||k||-1) sum_i d_i b^{k-e_i}               */
/*        + (||k||-1) sum_i b^{k-2e_i} = 0,   b^0 = 1/R,  d = x - y_c. */
/* ------------------------------------------------------------------ */
void orc_coulomb_coeffs(const double* d, int P, double* b)
{
    int n3 = (P + 1) * (P + 1) * (P + 1);
    for (int i = 0; i < n3; i++) b[i] = 0.0;
    double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    b[cube_idx(P, 0, 0, 0)] = 1.0 / sqrt(R2);
    for (int n = 1; n <= P; n++) {
        for (int k1 = n; k1 >= 0; k1--) {
            for (int k2 = n - k1; k2 >= 0; k2--) {
                int k3 = n - k1 - k2;
                double s1 = d[0] * cube_at(b, P, k1 - 1, k2, k3)
                          + d[1] * cube_at(b, P, k1, k2 - 1, k3)
                          + d[2] * cube_at(b, P, k1, k2, k3 - 1);
                double s2 = cube_at(b, P, k1 - 2, k2, k3)
                          + cube_at(b, P, k1, k2 - 2, k3)
                          + cube_at(b, P, k1, k2, k3 - 2);
                b[cube_idx(P, k1, k2, k3)] =
                    ((2.0 * n - 1.0) * s1 - (n - 1.0) * s2) / (n * R2);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Explicit Taylor coefficients (cross-check of the contracted form).  */
/* a^k_ij  from eq. (3.4); layout a[(9*?)...]: a[(3i+j)*n3 + idx(k)]  */
/* a~^k_ijl from eq. (3.7); layout t[(9i+3j+l)*n3 + idx(k)]           */
/* Both for ||k|| <= p; b is computed internally to order p+2.        */
/* ------------------------------------------------------------------ */
void orc_taylor_stokeslet(const double* d, int p, double* a)
{
    int P = p + 2, n3 = (p + 1) * (p + 1) * (p + 1);
    double* b = (double*)malloc(sizeof(double) * (P + 1) * (P + 1) * (P + 1));
    orc_coulomb_coeffs(d, P, b);
    for (int c = 0; c < 9 * n3; c++) a[c] = 0.0;
    for (int k1 = 0; k1 <= p; k1++)
        for (int k2 = 0; k1 + k2 <= p; k2++)
            for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                int k[3] = {k1, k2, k3};
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        int ei[3] = {0, 0, 0}, ej[3] = {0, 0, 0};
                        ei[i] = 1;
                        ej[j] = 1;
                        double dij = (i == j) ? 1.0 : 0.0;
                        double v = dij * cube_at(b, P, k1, k2, k3)
                                 + d[j] * (k[i] + 1) * cube_at(b, P, k1 + ei[0], k2 + ei[1], k3 + ei[2])
                                 - (k[i] + 1 - dij) * cube_at(b, P, k1 + ei[0] - ej[0], k2 + ei[1] - ej[1],
                                                              k3 + ei[2] - ej[2]);
                        a[(3 * i + j) * n3 + cube_idx(p, k1, k2, k3)] = v;
                    }
            }
    free(b);
}

void orc_taylor_stresslet(const double* d, int p, double* t)
{
    int P = p + 2, n3 = (p + 1) * (p + 1) * (p + 1);
    double* b = (double*)malloc(sizeof(double) * (P + 1) * (P + 1) * (P + 1));
    orc_coulomb_coeffs(d, P, b);
    for (int c = 0; c < 27 * n3; c++) t[c] = 0.0;
    for (int k1 = 0; k1 <= p; k1++)
        for (int k2 = 0; k1 + k2 <= p; k2++)
            for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                int k[3] = {k1, k2, k3};
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        for (int l = 0; l < 3; l++) {
                            int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                            double dij = (i == j), dil = (i == l), djl = (j == l);
                            /* b^{k+e_i+e_j} */
                            double b_ij = cube_at(b, P, k1 + e[i][0] + e[j][0], k2 + e[i][1] + e[j][1],
                                                  k3 + e[i][2] + e[j][2]);
                            /* b^{k+e_i+e_j-e_l} */
                            double b_ijl = cube_at(b, P, k1 + e[i][0] + e[j][0] - e[l][0],
                                                   k2 + e[i][1] + e[j][1] - e[l][1],
                                                   k3 + e[i][2] + e[j][2] - e[l][2]);
                            /* b^{k+e_l} */
                            double b_l = cube_at(b, P, k1 + e[l][0], k2 + e[l][1], k3 + e[l][2]);
                            double v = d[l] * (k[i] + 1) * (k[j] + 1 + dij) * b_ij
                                     - (k[i] + 1 - dil) * (k[j] + 1 + dij - djl) * b_ijl
                                     + dij * (k[l] + 1) * b_l;
                            t[(9 * i + 3 * j + l) * n3 + cube_idx(p, k1, k2, k3)] = v / 3.0;
                        }
            }
    free(b);
}

/* ------------------------------------------------------------------ */
/* Particle-cluster far field.                                         */
/* Moments of one cluster: Mf[j*n3 + idx(k)] = M_j^k (j = 0..2) and    */
/* Mt[(3j+l)*n3 + idx(k)] = M~_jl^k, cubes of order p.                 */
/* ------------------------------------------------------------------ */

/* Contracted evaluation, eqs. (4.4) S_final and (4.9) T_final. */
void orc_far_contracted(const double* d, int p, const double* Mf, const double* Mt, double* u)
{
    int P = p + 2, n3 = (p + 1) * (p + 1) * (p + 1);
    double* b = (double*)malloc(sizeof(double) * (P + 1) * (P + 1) * (P + 1));
    orc_coulomb_coeffs(d, P, b);
    int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double us[3] = {0, 0, 0}, ut[3] = {0, 0, 0};
    for (int k1 = 0; k1 <= p; k1++)
        for (int k2 = 0; k1 + k2 <= p; k2++)
            for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                int k[3] = {k1, k2, k3};
                int ik = cube_idx(p, k1, k2, k3);
                double M[3], Mtl[3][3];
                for (int j = 0; j < 3; j++) M[j] = Mf[j * n3 + ik];
                for (int j = 0; j < 3; j++)
                    for (int l = 0; l < 3; l++) Mtl[j][l] = Mt[(3 * j + l) * n3 + ik];
                /* Stokeslet, eq. (4.4) */
                double sigma = d[0] * M[0] + d[1] * M[1] + d[2] * M[2];
                for (int i = 0; i < 3; i++) {
                    double inner = cube_at(b, P, k1 + e[i][0], k2 + e[i][1], k3 + e[i][2]) * sigma;
                    for (int j = 0; j < 3; j++)
                        inner -= cube_at(b, P, k1 + e[i][0] - e[j][0], k2 + e[i][1] - e[j][1],
                                         k3 + e[i][2] - e[j][2]) * M[j];
                    us[i] += 2.0 * cube_at(b, P, k1, k2, k3) * M[i] + (k[i] + 1) * inner;
                }
                /* Stresslet, eq. (4.9) */
                double tau[3], mtr = Mtl[0][0] + Mtl[1][1] + Mtl[2][2];
                for (int j = 0; j < 3; j++) tau[j] = d[0] * Mtl[j][0] + d[1] * Mtl[j][1] + d[2] * Mtl[j][2];
                for (int i = 0; i < 3; i++) {
                    double t1 = 0.0, t2 = 0.0, t4 = 0.0;
                    for (int j = 0; j < 3; j++) {
                        double cj = k[j] + 1 + (i == j);
                        t1 += cj * cube_at(b, P, k1 + e[i][0] + e[j][0], k2 + e[i][1] + e[j][1],
                                           k3 + e[i][2] + e[j][2]) * tau[j];
                        for (int l = 0; l < 3; l++)
                            t2 += cj * cube_at(b, P, k1 + e[i][0] + e[j][0] - e[l][0],
                                               k2 + e[i][1] + e[j][1] - e[l][1],
                                               k3 + e[i][2] + e[j][2] - e[l][2]) * Mtl[j][l];
                        t4 += (k[j] + 1) * cube_at(b, P, k1 + e[j][0], k2 + e[j][1], k3 + e[j][2])
                            * (Mtl[i][j] + Mtl[j][i]);
                    }
                    double t3 = cube_at(b, P, k1 + e[i][0], k2 + e[i][1], k3 + e[i][2]) * mtr;
                    ut[i] += ((k[i] + 1) * t1 - (k[i] + 1) * t2 + (k[i] + 1) * t3 + t4) / 3.0;
                }
            }
    for (int i = 0; i < 3; i++) u[i] = us[i] + ut[i];
    free(b);
}

/* Explicit evaluation, eq. (2.9): sum_k a^k_ij M_j^k + a~^k_ijl M~_jl^k. */
void orc_far_explicit(const double* d, int p, const double* Mf, const double* Mt, double* u)
{
    int n3 = (p + 1) * (p + 1) * (p + 1);
    double* a = (double*)malloc(sizeof(double) * 9 * n3);
    double* t = (double*)malloc(sizeof(double) * 27 * n3);
    orc_taylor_stokeslet(d, p, a);
    orc_taylor_stresslet(d, p, t);
    for (int i = 0; i < 3; i++) {
        double s = 0.0;
        for (int ik = 0; ik < n3; ik++) {
            for (int j = 0; j < 3; j++) {
                s += a[(3 * i + j) * n3 + ik] * Mf[j * n3 + ik];
                for (int l = 0; l < 3; l++) s += t[(9 * i + 3 * j + l) * n3 + ik] * Mt[(3 * j + l) * n3 + ik];
            }
        }
        u[i] = s;
    }
    free(a);
    free(t);
}

/* ------------------------------------------------------------------ */
/* Taylor coefficients of G_nu(x, y) = (|x - y|^2 + eps^2)^(-nu) in y   */
/* about y_c, ||k|| <= P, nu = two_nu / 2.  Recurrence (3.2) follows    */
/* from R^2 D G = (x - y) G for G = 1/R; for G_nu, with                 */
/* s = |x - y|^2 + eps^2, the identity is s D_y G_nu = 2 nu (x - y) G_nu. */
/* Multiplying its Taylor series by t = y - y_c and summing over the    */
/* axes (the Euler operator takes t^k to ||k|| t^k) gives, with         */
/* d = x - y_c, n = ||k||, s_c = |d|^2 + eps^2:                         */
/*   n s_c c^k - (2n + 2nu - 2) sum_i d_i c^{k-e_i}                    */
/*                + (n + 2nu - 2) sum_i c^{k-2e_i} = 0,                 */
/* c^0 = s_c^(-nu); at nu = 1/2, eps = 0 it is (3.2).                   */
/* ------------------------------------------------------------------ */
void orc_coeffs_nu(const double* d, double eps, int two_nu, int P, double* c)
{
    int n3 = (P + 1) * (P + 1) * (P + 1);
    for (int i = 0; i < n3; i++) c[i] = 0.0;
    double sc = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps * eps;
    double nu2 = (double)two_nu;
    c[cube_idx(P, 0, 0, 0)] = pow(sc, -0.5 * nu2);
    for (int n = 1; n <= P; n++)
        for (int k1 = n; k1 >= 0; k1--)
            for (int k2 = n - k1; k2 >= 0; k2--) {
                int k3 = n - k1 - k2;
                double s1 = d[0] * cube_at(c, P, k1 - 1, k2, k3) + d[1] * cube_at(c, P, k1, k2 - 1, k3) +
                            d[2] * cube_at(c, P, k1, k2, k3 - 1);
                double s2 = cube_at(c, P, k1 - 2, k2, k3) + cube_at(c, P, k1, k2 - 2, k3) +
                            cube_at(c, P, k1, k2, k3 - 2);
                c[cube_idx(P, k1, k2, k3)] = ((2.0 * n + nu2 - 2.0) * s1 - (n + nu2 - 2.0) * s2) / (n * sc);
            }
}

/* Coefficient of t^k in prod_{a in ax[0..na)} (d_a - t_a) g(t), from the
 * coefficients g of g (product rule: every subset of the factors gives t). */
static double prod_coef(const double* g, int P, const int* k, const double* d, const int* ax, int na)
{
    double v = 0.0;
    for (int mask = 0; mask < (1 << na); mask++) {
        int kk[3] = {k[0], k[1], k[2]};
        double w = 1.0;
        for (int q = 0; q < na; q++) {
            if (mask & (1 << q)) {
                kk[ax[q]] -= 1;
                w = -w;
            } else {
                w *= d[ax[q]];
            }
        }
        v += w * cube_at(g, P, kk[0], kk[1], kk[2]);
    }
    return v;
}

/* Explicit Taylor coefficients of S^eps (layout of orc_taylor_stokeslet)
 * and T^eps (layout of orc_taylor_stresslet) in y about y_c, ||k|| <= p:
 * S^eps = delta_ij (G_1 + eps^2 G_3) + d_i d_j G_3 and
 * T^eps = d_i d_j d_l G_5 + (eps^2/2)(delta_ij d_l + delta_jl d_i + delta_il d_j) G_5,
 * G_m = s^(-m/2), each factor d_a = x_a - y_a = d_a(y_c) - t_a. */
void orc_taylor_stokeslet_reg(const double* d, double eps, int p, double* a)
{
    int n3 = (p + 1) * (p + 1) * (p + 1);
    double* g1 = (double*)malloc(sizeof(double) * n3);
    double* g3 = (double*)malloc(sizeof(double) * n3);
    orc_coeffs_nu(d, eps, 1, p, g1);
    orc_coeffs_nu(d, eps, 3, p, g3);
    for (int c = 0; c < 9 * n3; c++) a[c] = 0.0;
    for (int k1 = 0; k1 <= p; k1++)
        for (int k2 = 0; k1 + k2 <= p; k2++)
            for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                int k[3] = {k1, k2, k3}, ik = cube_idx(p, k1, k2, k3);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        int ax[2] = {i, j};
                        double v = prod_coef(g3, p, k, d, ax, 2);
                        if (i == j) v += g1[ik] + eps * eps * g3[ik];
                        a[(3 * i + j) * n3 + ik] = v;
                    }
            }
    free(g1);
    free(g3);
}

void orc_taylor_stresslet_reg(const double* d, double eps, int p, double* t)
{
    int n3 = (p + 1) * (p + 1) * (p + 1);
    double* g5 = (double*)malloc(sizeof(double) * n3);
    orc_coeffs_nu(d, eps, 5, p, g5);
    for (int c = 0; c < 27 * n3; c++) t[c] = 0.0;
    for (int k1 = 0; k1 <= p; k1++)
        for (int k2 = 0; k1 + k2 <= p; k2++)
            for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                int k[3] = {k1, k2, k3}, ik = cube_idx(p, k1, k2, k3);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        for (int l = 0; l < 3; l++) {
                            int a3[3] = {i, j, l};
                            double v = prod_coef(g5, p, k, d, a3, 3), w = 0.0;
                            if (i == j) w += prod_coef(g5, p, k, d, &a3[2], 1);
                            if (j == l) w += prod_coef(g5, p, k, d, &a3[0], 1);
                            if (i == l) w += prod_coef(g5, p, k, d, &a3[1], 1);
                            t[(9 * i + 3 * j + l) * n3 + ik] = v + 0.5 * eps * eps * w;
                        }
            }
    free(g5);
}

/* Regularized particle-cluster far field: eq. (2.9) with the regularized
 * kernels' Taylor coefficients, sum_k a^k_ij M_j^k + a~^k_ijl M~_jl^k. */
void orc_far_reg(const double* d, double eps, int p, const double* Mf, const double* Mt, double* u)
{
    int n3 = (p + 1) * (p + 1) * (p + 1);
    double* a = (double*)malloc(sizeof(double) * 9 * n3);
    double* t = (double*)malloc(sizeof(double) * 27 * n3);
    orc_taylor_stokeslet_reg(d, eps, p, a);
    orc_taylor_stresslet_reg(d, eps, p, t);
    for (int i = 0; i < 3; i++) {
        double sum = 0.0;
        for (int ik = 0; ik < n3; ik++)
            for (int j = 0; j < 3; j++) {
                sum += a[(3 * i + j) * n3 + ik] * Mf[j * n3 + ik];
                for (int l = 0; l < 3; l++) sum += t[(9 * i + 3 * j + l) * n3 + ik] * Mt[(3 * j + l) * n3 + ik];
            }
        u[i] = sum;
    }
    free(a);
    free(t);
}

/* Moments of a set of particles about yc (Section 2):                 */
/* M_j^k = sum_n (y^n - y_c)^k f_j^n,  M~_jl^k = sum_n (y^n-y_c)^k h_j^n nu_l^n */
void orc_moments(const double* y, const double* f, const double* h, const double* nu,
                 const int64_t* idx, int64_t count, const double* yc, int p, double* Mf, double* Mt)
{
    int n3 = (p + 1) * (p + 1) * (p + 1);
    for (int c = 0; c < 3 * n3; c++) Mf[c] = 0.0;
    for (int c = 0; c < 9 * n3; c++) Mt[c] = 0.0;
    for (int64_t q = 0; q < count; q++) {
        int64_t n = idx ? idx[q] : q;
        double px[ORC_PMAX + 1], py[ORC_PMAX + 1], pz[ORC_PMAX + 1];
        px[0] = py[0] = pz[0] = 1.0;
        for (int k = 1; k <= p; k++) {
            px[k] = px[k - 1] * (y[3 * n + 0] - yc[0]);
            py[k] = py[k - 1] * (y[3 * n + 1] - yc[1]);
            pz[k] = pz[k - 1] * (y[3 * n + 2] - yc[2]);
        }
        for (int k1 = 0; k1 <= p; k1++)
            for (int k2 = 0; k1 + k2 <= p; k2++)
                for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                    double mono = px[k1] * py[k2] * pz[k3];
                    int ik = cube_idx(p, k1, k2, k3);
                    for (int j = 0; j < 3; j++) Mf[j * n3 + ik] += mono * f[3 * n + j];
                    for (int j = 0; j < 3; j++)
                        for (int l = 0; l < 3; l++) Mt[(3 * j + l) * n3 + ik] += mono * h[3 * n + j] * nu[3 * n + l];
                }
    }
}

/* ------------------------------------------------------------------ */
/* Tree (Section 5).                                                   */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t begin, count; /* range in tree->order */
    int level;
    int64_t cell[3];      /* integer cell coordinates at this level */
    int nchild;
    int64_t child[8];
    double yc[3];
    double rc2;           /* max squared distance centre -> particle */
} orc_node;

typedef struct {
    int64_t N;
    int N0, shrink;
    const double* x;      /* caller's positions, row-major (N,3); kept by pointer */
    double lo[3], side;
    uint32_t* q;          /* quantised coordinates (N,3) */
    int64_t* order;       /* particle indices, grouped by node */
    orc_node* nodes;
    int64_t nnodes, cap;
    int p;                /* order of stored moments, -1 if none */
    double* Mf;           /* nnodes * 3 * n3 */
    double* Mt;           /* nnodes * 9 * n3 */
    const double *f, *h, *nu;
} orc_tree;

static int64_t new_node(orc_tree* t)
{
    if (t->nnodes == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 64;
        t->nodes = (orc_node*)realloc(t->nodes, sizeof(orc_node) * t->cap);
    }
    memset(&t->nodes[t->nnodes], 0, sizeof(orc_node));
    return t->nnodes++;
}

/* Build the subtree over order[begin, begin+count) for the cell at `level`. */
static void build_rec(orc_tree* t, int64_t id)
{
    orc_node nd = t->nodes[id];
    if (nd.count <= t->N0 || nd.level >= ORC_MAXDEPTH) return;
    int shift = ORC_MAXDEPTH - nd.level - 1; /* bit that selects the child */
    /* stable partition of the node's particles into 8 octants */
    int64_t cnt[8] = {0};
    for (int64_t q = 0; q < nd.count; q++) {
        int64_t n = t->order[nd.begin + q];
        int oct = (int)(((t->q[3 * n + 0] >> shift) & 1u) << 2 | ((t->q[3 * n + 1] >> shift) & 1u) << 1 |
                        ((t->q[3 * n + 2] >> shift) & 1u));
        cnt[oct]++;
    }
    int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * (size_t)nd.count);
    int64_t start[8], pos[8];
    start[0] = 0;
    for (int o = 1; o < 8; o++) start[o] = start[o - 1] + cnt[o - 1];
    for (int o = 0; o < 8; o++) pos[o] = start[o];
    for (int64_t q = 0; q < nd.count; q++) {
        int64_t n = t->order[nd.begin + q];
        int oct = (int)(((t->q[3 * n + 0] >> shift) & 1u) << 2 | ((t->q[3 * n + 1] >> shift) & 1u) << 1 |
                        ((t->q[3 * n + 2] >> shift) & 1u));
        tmp[pos[oct]++] = n;
    }
    memcpy(t->order + nd.begin, tmp, sizeof(int64_t) * (size_t)nd.count);
    free(tmp);
    for (int o = 0; o < 8; o++) {
        if (cnt[o] == 0) continue;
        int64_t c = new_node(t);
        orc_node* ch = &t->nodes[c];
        ch->begin = nd.begin + start[o];
        ch->count = cnt[o];
        ch->level = nd.level + 1;
        ch->cell[0] = 2 * nd.cell[0] + ((o >> 2) & 1);
        ch->cell[1] = 2 * nd.cell[1] + ((o >> 1) & 1);
        ch->cell[2] = 2 * nd.cell[2] + (o & 1);
        orc_node* par = &t->nodes[id];
        par->child[par->nchild++] = c;
    }
    int nch = t->nodes[id].nchild;
    for (int c = 0; c < nch; c++) build_rec(t, t->nodes[id].child[c]);
}

static void node_geometry(orc_tree* t, orc_node* nd)
{
    const double* x = t->x;
    if (t->shrink) {
        double mn[3], mx[3];
        for (int a = 0; a < 3; a++) {
            mn[a] = INFINITY;
            mx[a] = -INFINITY;
        }
        for (int64_t q = 0; q < nd->count; q++) {
            int64_t n = t->order[nd->begin + q];
            for (int a = 0; a < 3; a++) {
                if (x[3 * n + a] < mn[a]) mn[a] = x[3 * n + a];
                if (x[3 * n + a] > mx[a]) mx[a] = x[3 * n + a];
            }
        }
        for (int a = 0; a < 3; a++) nd->yc[a] = (mn[a] + mx[a]) * 0.5;
    } else {
        double cs = ldexp(t->side, -nd->level);
        for (int a = 0; a < 3; a++) nd->yc[a] = t->lo[a] + ((double)nd->cell[a] + 0.5) * cs;
    }
    double r2 = 0.0;
    for (int64_t q = 0; q < nd->count; q++) {
        int64_t n = t->order[nd->begin + q];
        double dx = x[3 * n + 0] - nd->yc[0], dy = x[3 * n + 1] - nd->yc[1], dz = x[3 * n + 2] - nd->yc[2];
        double s = (dx * dx + dy * dy) + dz * dz;
        if (s > r2) r2 = s;
    }
    nd->rc2 = r2;
}

/* Root cube and quantised coordinates (Section 5). */
orc_tree* orc_tree_build(const double* x, int64_t N, int N0, int shrink)
{
    if (N < 1 || N0 < 1) return NULL;
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->N = N;
    t->N0 = N0;
    t->shrink = shrink;
    t->x = x;
    t->p = -1;
    double hi[3];
    for (int a = 0; a < 3; a++) {
        t->lo[a] = x[a];
        hi[a] = x[a];
    }
    for (int64_t n = 1; n < N; n++)
        for (int a = 0; a < 3; a++) {
            if (x[3 * n + a] < t->lo[a]) t->lo[a] = x[3 * n + a];
            if (x[3 * n + a] > hi[a]) hi[a] = x[3 * n + a];
        }
    t->side = 0.0;
    for (int a = 0; a < 3; a++)
        if (hi[a] - t->lo[a] > t->side) t->side = hi[a] - t->lo[a];
    double scale = t->side > 0.0 ? 2097152.0 / t->side : 0.0; /* 2^21 cells per axis */
    t->q = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)N);
    t->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t n = 0; n < N; n++) {
        t->order[n] = n;
        for (int a = 0; a < 3; a++) {
            double v = floor((x[3 * n + a] - t->lo[a]) * scale);
            if (v > 2097151.0) v = 2097151.0;
            t->q[3 * n + a] = (uint32_t)v;
        }
    }
    int64_t root = new_node(t);
    t->nodes[root].begin = 0;
    t->nodes[root].count = N;
    t->nodes[root].level = 0;
    build_rec(t, root);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->nnodes; c++) node_geometry(t, &t->nodes[c]);
    return t;
}

void orc_tree_free(orc_tree* t)
{
    if (!t) return;
    free(t->q);
    free(t->order);
    free(t->nodes);
    free(t->Mf);
    free(t->Mt);
    free(t);
}

int64_t orc_tree_num_nodes(const orc_tree* t) { return t->nnodes; }

void orc_tree_root(const orc_tree* t, double* lo, double* side)
{
    for (int a = 0; a < 3; a++) lo[a] = t->lo[a];
    *side = t->side;
}

/* Export per-node records; any pointer may be NULL. */
void orc_tree_export(const orc_tree* t, int64_t* begin, int64_t* count, int32_t* level, int64_t* cell,
                     int32_t* nchild, int64_t* child, double* yc, double* rc2)
{
    for (int64_t c = 0; c < t->nnodes; c++) {
        const orc_node* nd = &t->nodes[c];
        if (begin) begin[c] = nd->begin;
        if (count) count[c] = nd->count;
        if (level) level[c] = nd->level;
        if (cell)
            for (int a = 0; a < 3; a++) cell[3 * c + a] = nd->cell[a];
        if (nchild) nchild[c] = nd->nchild;
        if (child)
            for (int o = 0; o < 8; o++) child[8 * c + o] = o < nd->nchild ? nd->child[o] : -1;
        if (yc)
            for (int a = 0; a < 3; a++) yc[3 * c + a] = nd->yc[a];
        if (rc2) rc2[c] = nd->rc2;
    }
}

void orc_tree_order(const orc_tree* t, int64_t* order) { memcpy(order, t->order, sizeof(int64_t) * t->N); }

void orc_tree_quantized(const orc_tree* t, uint32_t* q) { memcpy(q, t->q, sizeof(uint32_t) * 3 * t->N); }

/* Cluster moments for every node (Section 2), from their definition. */
int orc_tree_moments(orc_tree* t, const double* f, const double* h, const double* nu, int p)
{
    if (p < 0 || p > ORC_PMAX) return -1;
    int n3 = (p + 1) * (p + 1) * (p + 1);
    free(t->Mf);
    free(t->Mt);
    t->Mf = (double*)malloc(sizeof(double) * 3 * n3 * (size_t)t->nnodes);
    t->Mt = (double*)malloc(sizeof(double) * 9 * n3 * (size_t)t->nnodes);
    t->f = f;
    t->h = h;
    t->nu = nu;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->nnodes; c++) {
        const orc_node* nd = &t->nodes[c];
        orc_moments(t->x, f, h, nu, t->order + nd->begin, nd->count, nd->yc, p, t->Mf + (size_t)c * 3 * n3,
                    t->Mt + (size_t)c * 9 * n3);
    }
    t->p = p;
    return 0;
}

void orc_tree_export_moments(const orc_tree* t, int64_t node, double* Mf, double* Mt)
{
    int n3 = (t->p + 1) * (t->p + 1) * (t->p + 1);
    memcpy(Mf, t->Mf + (size_t)node * 3 * n3, sizeof(double) * 3 * n3);
    memcpy(Mt, t->Mt + (size_t)node * 9 * n3, sizeof(double) * 9 * n3);
}

/* ------------------------------------------------------------------ */
/* Per-target interaction set (Section 5, MAC of eq. 5.1).             */
/*                                                                     */
/* Starting from the root, a cluster C is accepted for the far-field   */
/* approximation when the target sees it under r/R <= theta; a leaf    */
/* that is not accepted is summed directly; any other cluster that is  */
/* not accepted is replaced by its children.  The walk below keeps the */
/* clusters still to be examined on an explicit stack (children pushed */
/* in reverse octant order, so they are examined in octant order) and  */
/* records every decision in an interaction list, in the order the     */
/* decisions are made.  The velocity is then the sum over that list.   */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t node;
    int far; /* 1: far-field approximation, 0: direct sum over the leaf */
} orc_entry;

/* Interaction list of the target at xd.  list has room for every node;
 * returns the number of entries. */
static int64_t interaction_list(const orc_tree* t, const double* xd, double theta, orc_entry* list, int64_t* stack)
{
    int64_t nlist = 0, top = 0;
    stack[top++] = 0;
    while (top > 0) {
        const int64_t c = stack[--top];
        const orc_node* nd = &t->nodes[c];
        double d[3] = {xd[0] - nd->yc[0], xd[1] - nd->yc[1], xd[2] - nd->yc[2]};
        double R2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        if ((R2 > 0.0) && (nd->rc2 <= (theta * theta) * R2)) {
            list[nlist].node = c;
            list[nlist].far = 1;
            nlist++;
        } else if (nd->nchild == 0) {
            list[nlist].node = c;
            list[nlist].far = 0;
            nlist++;
        } else {
            for (int o = nd->nchild - 1; o >= 0; o--) stack[top++] = nd->child[o];
        }
    }
    return nlist;
}

/* Direct sum of one leaf at xm in the contracted form of Section 4.1:
 * u_i += f_i/r + d_i (s + t), s = (d.f)/r^3, t = (d.h)(d.nu)/r^5, with the
 * leaf's sources at positions y (row-major), pairs with r == 0 skipped. */
static void leaf_direct(const orc_tree* t, const orc_node* nd, const double* y_all, const double* f_all,
                        const double* h_all, const double* nu_all, const double* xm, double* u)
{
    for (int64_t q = 0; q < nd->count; q++) {
        int64_t n = t->order[nd->begin + q];
        const double* y = y_all + 3 * n;
        double d[3] = {xm[0] - y[0], xm[1] - y[1], xm[2] - y[2]};
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 == 0.0) continue;
        double r = sqrt(r2);
        const double* f = f_all + 3 * n;
        const double* h = h_all + 3 * n;
        const double* nu = nu_all + 3 * n;
        double s = (d[0] * f[0] + d[1] * f[1] + d[2] * f[2]) / (r * r2);
        double tt = (d[0] * h[0] + d[1] * h[1] + d[2] * h[2]) * (d[0] * nu[0] + d[1] * nu[1] + d[2] * nu[2]) /
                    (r2 * r2 * r);
        for (int i = 0; i < 3; i++) u[i] += f[i] / r + d[i] * (s + tt);
    }
}

/* Direct sum of one leaf at xm with the regularized kernels formed
 * explicitly (orc_stokeslet_reg, orc_stresslet_reg), r == 0 skipped. */
static void leaf_direct_reg(const orc_tree* t, const orc_node* nd, const double* y_all, const double* f_all,
                            const double* h_all, const double* nu_all, double eps, const double* xm, double* u)
{
    for (int64_t q = 0; q < nd->count; q++) {
        int64_t n = t->order[nd->begin + q];
        const double* y = y_all + 3 * n;
        if (xm[0] == y[0] && xm[1] == y[1] && xm[2] == y[2]) continue;
        double S[9], T[27];
        orc_stokeslet_reg(xm, y, eps, S);
        orc_stresslet_reg(xm, y, eps, T);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                u[i] += S[3 * i + j] * f_all[3 * n + j];
                for (int l = 0; l < 3; l++) u[i] += T[9 * i + 3 * j + l] * h_all[3 * n + j] * nu_all[3 * n + l];
            }
    }
}

/* Far field of cluster moments stored at order P (cubes Mf: 3 x (P+1)^3,
 * Mt: 9 x (P+1)^3), evaluated at order p <= P by eqs. (4.4) + (4.9), or
 * for eps > 0 by the regularized expansion (orc_far_reg). */
static void far_at_order(const double* d, int p, int P, const double* MfP, const double* MtP, double eps,
                         double* uf)
{
    if (p == P) {
        if (eps > 0.0)
            orc_far_reg(d, eps, p, MfP, MtP, uf);
        else
            orc_far_contracted(d, p, MfP, MtP, uf);
        return;
    }
    int N3 = (P + 1) * (P + 1) * (P + 1), m3 = (p + 1) * (p + 1) * (p + 1);
    double* Mf = (double*)malloc(sizeof(double) * 3 * m3);
    double* Mt = (double*)malloc(sizeof(double) * 9 * m3);
    for (int comp = 0; comp < 12; comp++)
        for (int k1 = 0; k1 <= p; k1++)
            for (int k2 = 0; k2 <= p; k2++)
                for (int k3 = 0; k3 <= p; k3++) {
                    double v = 0.0;
                    if (k1 + k2 + k3 <= p)
                        v = comp < 3 ? MfP[comp * N3 + cube_idx(P, k1, k2, k3)]
                                     : MtP[(comp - 3) * N3 + cube_idx(P, k1, k2, k3)];
                    if (comp < 3)
                        Mf[comp * m3 + cube_idx(p, k1, k2, k3)] = v;
                    else
                        Mt[(comp - 3) * m3 + cube_idx(p, k1, k2, k3)] = v;
                }
    if (eps > 0.0)
        orc_far_reg(d, eps, p, Mf, Mt, uf);
    else
        orc_far_contracted(d, p, Mf, Mt, uf);
    free(Mf);
    free(Mt);
}

typedef struct {
    int64_t nfar, nnear_leaves, nnear_pairs;
} orc_counts;

/* What a sum over an interaction list reads: source positions and weights,
 * per-node moments of order P about the nodes' centres, evaluation order p. */
typedef struct {
    const orc_tree* t;
    const double *x, *f, *h, *nu;
    const double *Mf, *Mt;
    int P, p;
    double eps; /* > 0: regularized kernels */
} orc_sources;

/* u at xm = sum over the interaction list, in list order: far entries by
 * eqs. (4.4) + (4.9) at d = xm - y_c, near entries by Section 4.1. */
static void sum_interactions(const orc_sources* s, const orc_entry* list, int64_t nlist, const double* xm, double* u,
                             orc_counts* cnt)
{
    const int64_t N3 = (int64_t)(s->P + 1) * (s->P + 1) * (s->P + 1);
    for (int64_t e = 0; e < nlist; e++) {
        const orc_node* nd = &s->t->nodes[list[e].node];
        if (list[e].far) {
            double d[3] = {xm[0] - nd->yc[0], xm[1] - nd->yc[1], xm[2] - nd->yc[2]}, uf[3];
            far_at_order(d, s->p, s->P, s->Mf + (size_t)list[e].node * 3 * N3, s->Mt + (size_t)list[e].node * 9 * N3,
                         s->eps, uf);
            for (int i = 0; i < 3; i++) u[i] += uf[i];
            if (cnt) cnt->nfar++;
        } else {
            if (s->eps > 0.0)
                leaf_direct_reg(s->t, nd, s->x, s->f, s->h, s->nu, s->eps, xm, u);
            else
                leaf_direct(s->t, nd, s->x, s->f, s->h, s->nu, xm, u);
            if (cnt) {
                cnt->nnear_leaves++;
                cnt->nnear_pairs += nd->count;
            }
        }
    }
}

/* Treecode velocity at M targets tx (row-major (M,3)): the interaction list
 * of each target (decided at the target), then its sum, with the kernels of
 * eqs. (1.2a,b) (eps = 0) or the regularized ones (eps > 0; same tree, MAC,
 * moments and lists).  Requires moments of order >= p.  Optional per-target
 * counters (may be NULL). Returns 0 or -1. */
int orc_treecode_eps(const orc_tree* t, const double* tx, int64_t M, double theta, int p, double eps, double* u,
                     int64_t* nfar, int64_t* nnear_leaves, int64_t* nnear_pairs, int nthreads)
{
    if (t->p < 0 || p > t->p || p < 0 || eps < 0.0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    const orc_sources s = {t, t->x, t->f, t->h, t->nu, t->Mf, t->Mt, t->p, p, eps};
#pragma omp parallel
    {
        orc_entry* list = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)t->nnodes);
        int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)t->nnodes);
#pragma omp for schedule(dynamic, 4)
        for (int64_t m = 0; m < M; m++) {
            double acc[3] = {0, 0, 0};
            orc_counts cnt = {0, 0, 0};
            const int64_t n = interaction_list(t, tx + 3 * m, theta, list, stack);
            sum_interactions(&s, list, n, tx + 3 * m, acc, &cnt);
            for (int i = 0; i < 3; i++) u[3 * m + i] = acc[i];
            if (nfar) nfar[m] = cnt.nfar;
            if (nnear_leaves) nnear_leaves[m] = cnt.nnear_leaves;
            if (nnear_pairs) nnear_pairs[m] = cnt.nnear_pairs;
        }
        free(list);
        free(stack);
    }
    return 0;
}

int orc_treecode(const orc_tree* t, const double* tx, int64_t M, double theta, int p, double* u, int64_t* nfar,
                 int64_t* nnear_leaves, int64_t* nnear_pairs, int nthreads)
{
    return orc_treecode_eps(t, tx, M, theta, p, 0.0, u, nfar, nnear_leaves, nnear_pairs, nthreads);
}

/* Sum of the counts of the far clusters of each target (partition check). */
void orc_far_mass(const orc_tree* t, const double* tx, int64_t M, double theta, int64_t* mass)
{
#pragma omp parallel
    {
        orc_entry* list = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)t->nnodes);
        int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)t->nnodes);
#pragma omp for schedule(dynamic, 16)
        for (int64_t m = 0; m < M; m++) {
            const int64_t n = interaction_list(t, tx + 3 * m, theta, list, stack);
            int64_t s = 0;
            for (int64_t e = 0; e < n; e++)
                if (list[e].far) s += t->nodes[list[e].node].count;
            mass[m] = s;
        }
        free(list);
        free(stack);
    }
}

/* Threads of every later parallel region (n >= 1). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#endif
    (void)n;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Frozen-structure evaluation, for finite-difference checks of the    */
/* adjoint.  The tree built from the original positions keeps its      */
/* cluster membership, centres y_c and radii; every target's           */
/* interaction list is decided at its decision position td; the        */
/* moments (Section 2) and the direct sums (Section 4.1) use the moved  */
/* source positions xe, and far fields and direct sums are evaluated   */
/* at the moved target positions te.  With xe = x and td = te this is  */
/* orc_treecode.                                                       */
/* ------------------------------------------------------------------ */
int orc_treecode_frozen(const orc_tree* t, const double* xe, const double* f, const double* h, const double* nu, int p,
                        const double* td, const double* te, int64_t M, double theta, double* u, int nthreads)
{
    if (p < 0 || p > ORC_PMAX) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    int n3 = (p + 1) * (p + 1) * (p + 1);
    double* Mf = (double*)malloc(sizeof(double) * 3 * n3 * (size_t)t->nnodes);
    double* Mt = (double*)malloc(sizeof(double) * 9 * n3 * (size_t)t->nnodes);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->nnodes; c++) {
        const orc_node* nd = &t->nodes[c];
        orc_moments(xe, f, h, nu, t->order + nd->begin, nd->count, nd->yc, p, Mf + (size_t)c * 3 * n3,
                    Mt + (size_t)c * 9 * n3);
    }
    const orc_sources s = {t, xe, f, h, nu, Mf, Mt, p, p, 0.0};
#pragma omp parallel
    {
        orc_entry* list = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)t->nnodes);
        int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)t->nnodes);
#pragma omp for schedule(dynamic, 4)
        for (int64_t m = 0; m < M; m++) {
            double acc[3] = {0, 0, 0};
            const int64_t n = interaction_list(t, td + 3 * m, theta, list, stack);
            sum_interactions(&s, list, n, te + 3 * m, acc, NULL);
            for (int i = 0; i < 3; i++) u[3 * m + i] = acc[i];
        }
        free(list);
        free(stack);
    }
    free(Mf);
    free(Mt);
    return 0;
}
