/*
 * FP64 kernel sums for the oracle (test infrastructure only; never part of the product path).
 *
 * One routine: for every target group g, for every target i of that group and every source j
 * in the group's source ranges, add K(x_i, y_j) s_j to f_i, where K is the 3D Laplace kernel
 * 1/(4 pi |x - y|) (Eq. 2, normalised by 4 pi) or, with kappa > 0, the modified Helmholtz
 * (Yukawa) kernel exp(-kappa |x - y|) / (4 pi |x - y|), i.e. Eq. 1 restricted to the given
 * pairs.  Pairs with |x_i - y_j| == 0 exactly are skipped: that excludes self-interaction and
 * coincident points.  With `grad` non-NULL the gradient with respect to the target position,
 * -sum_j s_j (1 + kappa r) exp(-kappa r) (x_i - y_j) / (4 pi r^3), r = |x_i - y_j|, is
 * accumulated as well.
 *
 * This is a plain double loop with no blocking; OpenMP only splits the groups between threads.
 */
#include <math.h>
#include <stdint.h>

#define INV4PI 0.079577471545947667884441881686257181  /* 1/(4 pi) */

void oracle_grouped_sum(int64_t n_groups,
                        const int64_t *t_off,      /* [n_groups+1]: targets of group g are t_off[g]..t_off[g+1]-1 */
                        const double *tx,          /* [n_targets*3] target coordinates */
                        const int64_t *r_off,      /* [n_groups+1]: source ranges of group g are r_off[g]..r_off[g+1]-1 */
                        const int64_t *ranges,     /* [n_ranges*2]: (begin, end) into the source arrays */
                        const double *sx,          /* [n_sources*3] source coordinates */
                        const double *sq,          /* [n_sources] source densities */
                        double *pot,               /* [n_targets], accumulated */
                        double *grad,              /* [n_targets*3] or NULL, accumulated */
                        double kappa)              /* 0: Laplace; > 0: Yukawa decay rate */
{
    int64_t g;
#pragma omp parallel for schedule(dynamic, 1)
    for (g = 0; g < n_groups; ++g) {
        for (int64_t i = t_off[g]; i < t_off[g + 1]; ++i) {
            const double xi = tx[3 * i], yi = tx[3 * i + 1], zi = tx[3 * i + 2];
            double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
            for (int64_t r = r_off[g]; r < r_off[g + 1]; ++r) {
                for (int64_t j = ranges[2 * r]; j < ranges[2 * r + 1]; ++j) {
                    const double dx = xi - sx[3 * j];
                    const double dy = yi - sx[3 * j + 1];
                    const double dz = zi - sx[3 * j + 2];
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0) continue;
                    const double rinv = 1.0 / sqrt(r2);
                    const double r = r2 * rinv;
                    const double e = kappa > 0.0 ? exp(-kappa * r) : 1.0;
                    const double w = sq[j] * rinv * e;
                    f += w;
                    if (grad) {
                        const double w3 = w * (1.0 + kappa * r) * rinv * rinv;
                        gx -= w3 * dx;
                        gy -= w3 * dy;
                        gz -= w3 * dz;
                    }
                }
            }
            pot[i] += f * INV4PI;
            if (grad) {
                grad[3 * i] += gx * INV4PI;
                grad[3 * i + 1] += gy * INV4PI;
                grad[3 * i + 2] += gz * INV4PI;
            }
        }
    }
}

/*
 * The same sums with the Helmholtz kernel exp(i k |x - y|) / (4 pi |x - y|) and complex densities.
 * Complex arrays are interleaved (re, im): sq[2 * n_sources], pot[2 * n_targets] and, with grad
 * non-NULL, grad[6 * n_targets] = (d/dx re, d/dx im, d/dy re, d/dy im, d/dz re, d/dz im) per target.
 * Per pair, w = s_j exp(i k r) / r and the gradient term is w (i k r - 1) (x_i - y_j) / r^2.
 */
void oracle_grouped_sum_helm(int64_t n_groups, const int64_t *t_off, const double *tx, const int64_t *r_off,
                             const int64_t *ranges, const double *sx, const double *sq, double *pot, double *grad,
                             double k)
{
    int64_t g;
#pragma omp parallel for schedule(dynamic, 1)
    for (g = 0; g < n_groups; ++g) {
        for (int64_t i = t_off[g]; i < t_off[g + 1]; ++i) {
            const double xi = tx[3 * i], yi = tx[3 * i + 1], zi = tx[3 * i + 2];
            double fr = 0.0, fi = 0.0;
            double gr[3] = {0.0, 0.0, 0.0}, gi[3] = {0.0, 0.0, 0.0};
            for (int64_t r = r_off[g]; r < r_off[g + 1]; ++r) {
                for (int64_t j = ranges[2 * r]; j < ranges[2 * r + 1]; ++j) {
                    const double d[3] = {xi - sx[3 * j], yi - sx[3 * j + 1], zi - sx[3 * j + 2]};
                    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 == 0.0) continue;
                    const double rinv = 1.0 / sqrt(r2);
                    const double rr = r2 * rinv;
                    const double c = cos(k * rr), s = sin(k * rr);
                    const double qr = sq[2 * j], qi = sq[2 * j + 1];
                    const double wr = (qr * c - qi * s) * rinv, wi = (qr * s + qi * c) * rinv;
                    fr += wr;
                    fi += wi;
                    if (grad) {
                        /* w (i k r - 1) / r^2 */
                        const double zr = (-wr - k * rr * wi) * rinv * rinv;
                        const double zi = (-wi + k * rr * wr) * rinv * rinv;
                        for (int a = 0; a < 3; ++a) {
                            gr[a] += zr * d[a];
                            gi[a] += zi * d[a];
                        }
                    }
                }
            }
            pot[2 * i] += fr * INV4PI;
            pot[2 * i + 1] += fi * INV4PI;
            if (grad)
                for (int a = 0; a < 3; ++a) {
                    grad[6 * i + 2 * a] += gr[a] * INV4PI;
                    grad[6 * i + 2 * a + 1] += gi[a] * INV4PI;
                }
        }
    }
}

/* Number of threads OpenMP would use (1 when built without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
