/*
 * FP64 short-range pair sums of the P3M oracle -- test infrastructure only.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg load this library.
 * It shares no code with the CUDA path.
 *
 * The short-range acceleration of particle i (textbook P3M with the Gaussian force split
 * used by the guide's P3M kick algorithm, Ch. Parameters, "PM_scale" and "P3M_cutoff"):
 *
 *   a_SR,i = sum_{j != i, 0 < r_ij < r_c}  Gm * g(r_ij / r_s) * d_ij / (r_ij^2 + eps^2)^(3/2)
 *
 *   d_ij = x_j - x_i reduced to the minimum periodic image, r_ij = |d_ij|,
 *   g(x) = erfc(x/2) + x/sqrt(pi) * exp(-x^2/4),
 *
 * eps being the Plummer softening radius (Ch. Parameters, "softeningfactors").  Pairs with
 * r_ij = 0 contribute nothing (their displacement is zero) and are skipped so that eps = 0
 * stays finite.  Plain loops over particles, OpenMP over the target particles only (each
 * target's sum runs serially in a fixed order, so results do not depend on the thread count).
 */
#include <math.h>
#include <stdint.h>

static double min_image(double d, double box)
{
    if (d > 0.5 * box) d -= box;
    else if (d < -0.5 * box) d += box;
    return d;
}

static double g_split(double x)
{
    const double inv_sqrt_pi = 0.56418958354775628695;
    return erfc(0.5 * x) + x * inv_sqrt_pi * exp(-0.25 * x * x);
}

/* Adds the pair term of j on i into acc[0..2]; returns 1 when the pair is inside the cutoff. */
static int pair_term(const double *pos, int64_t n, int64_t i, int64_t j, double box,
                     double r_s, double r_c, double eps, double gm, double *acc)
{
    double dx = min_image(pos[j] - pos[i], box);
    double dy = min_image(pos[n + j] - pos[n + i], box);
    double dz = min_image(pos[2 * n + j] - pos[2 * n + i], box);
    double r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < r_c * r_c) || r2 == 0.0) return 0;
    double r = sqrt(r2);
    double s2 = r2 + eps * eps;
    double f = gm * g_split(r / r_s) / (s2 * sqrt(s2));
    acc[0] += f * dx;
    acc[1] += f * dy;
    acc[2] += f * dz;
    return 1;
}

/*
 * Chaining-cell version: the neighbours of a particle are the particles of the 27 cells
 * around its own cell (periodic), n_c >= 3 cells per side of width box/n_c >= r_c.
 *   cell_of[i]    cell id of particle i, (cz*n_c + cy)*n_c + cx
 *   order[k]      particle indices sorted by cell id
 *   cell_start[c] first position in `order` of cell c, cell_start[n_c^3] = n
 *   targets       particles whose acceleration is wanted (NULL: all n)
 * acc is SoA [3][n_targets] and is overwritten; *n_pairs receives the number of ordered
 * pairs (target, j) inside the cutoff.
 */
void sr_accel_cells(int64_t n, const double *pos, double box, int64_t n_c,
                    const int64_t *cell_of, const int64_t *order, const int64_t *cell_start,
                    double r_s, double r_c, double eps, double gm,
                    const int64_t *targets, int64_t n_targets, double *acc, int64_t *n_pairs)
{
    int64_t nt = targets ? n_targets : n;
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : pairs)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        int64_t c = cell_of[i];
        int64_t cx = c % n_c, cy = (c / n_c) % n_c, cz = c / (n_c * n_c);
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t oz = -1; oz <= 1; ++oz)
            for (int64_t oy = -1; oy <= 1; ++oy)
                for (int64_t ox = -1; ox <= 1; ++ox) {
                    int64_t nx = (cx + ox + n_c) % n_c;
                    int64_t ny = (cy + oy + n_c) % n_c;
                    int64_t nz = (cz + oz + n_c) % n_c;
                    int64_t nc = (nz * n_c + ny) * n_c + nx;
                    for (int64_t k = cell_start[nc]; k < cell_start[nc + 1]; ++k) {
                        int64_t j = order[k];
                        if (j == i) continue;
                        pairs += pair_term(pos, n, i, j, box, r_s, r_c, eps, gm, a);
                    }
                }
        acc[t] = a[0];
        acc[nt + t] = a[1];
        acc[2 * nt + t] = a[2];
    }
    *n_pairs = pairs;
}

/* All-pairs version of the same sum (minimum image, r_c < box/2): the brute-force check. */
void sr_accel_brute(int64_t n, const double *pos, double box, double r_s, double r_c,
                    double eps, double gm, const int64_t *targets, int64_t n_targets,
                    double *acc, int64_t *n_pairs)
{
    int64_t nt = targets ? n_targets : n;
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            pairs += pair_term(pos, n, i, j, box, r_s, r_c, eps, gm, a);
        }
        acc[t] = a[0];
        acc[nt + t] = a[1];
        acc[2 * nt + t] = a[2];
    }
    *n_pairs = pairs;
}

/* Number of OpenMP threads the loops above use (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Transposed Jacobian of the short-range accelerations applied to a vector field v (the
 * reverse-mode derivative used by the adjoint of the step):
 *   out_k = sum_{j in the 27 cells, 0 < r_kj < r_c} J(d_kj) (v_j - v_k),
 *   J(d) = h(r) I + (h'(r)/r) d d^T,  h(r) = Gm g(r/r_s) / (r^2 + eps^2)^(3/2),
 *   h'(r) = Gm [g'(r/r_s)/r_s (r^2+eps^2)^(-3/2) - 3 r g(r/r_s) (r^2+eps^2)^(-5/2)],
 *   g'(x) = -x^2 exp(-x^2/4) / (2 sqrt(pi)).
 * (J is even in d, so the contributions of k as the i and as the j of a pair combine into
 * this single sum.)  v and out are SoA [3][n]; same cell arguments as sr_accel_cells.
 */
void sr_vjp_cells(int64_t n, const double *pos, const double *v, double box, int64_t n_c,
                  const int64_t *cell_of, const int64_t *order, const int64_t *cell_start,
                  double r_s, double r_c, double eps, double gm, double *out)
{
    const double inv_sqrt_pi = 0.56418958354775628695;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
        int64_t c = cell_of[k];
        int64_t cx = c % n_c, cy = (c / n_c) % n_c, cz = c / (n_c * n_c);
        double o[3] = {0.0, 0.0, 0.0};
        for (int64_t oz = -1; oz <= 1; ++oz)
            for (int64_t oy = -1; oy <= 1; ++oy)
                for (int64_t ox = -1; ox <= 1; ++ox) {
                    int64_t nc = ((((cz + oz + n_c) % n_c) * n_c + (cy + oy + n_c) % n_c) * n_c +
                                  (cx + ox + n_c) % n_c);
                    for (int64_t t = cell_start[nc]; t < cell_start[nc + 1]; ++t) {
                        int64_t j = order[t];
                        if (j == k) continue;
                        double d[3] = {min_image(pos[j] - pos[k], box),
                                       min_image(pos[n + j] - pos[n + k], box),
                                       min_image(pos[2 * n + j] - pos[2 * n + k], box)};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(r2 < r_c * r_c) || r2 == 0.0) continue;
                        double r = sqrt(r2), x = r / r_s, s2 = r2 + eps * eps;
                        double s3 = s2 * sqrt(s2);
                        double g = g_split(x);
                        double gp = -x * x * exp(-0.25 * x * x) * 0.5 * inv_sqrt_pi;
                        double h = gm * g / s3;
                        double hp = gm * (gp / r_s / s3 - 3.0 * r * g / (s3 * s2));
                        double w[3] = {v[j] - v[k], v[n + j] - v[n + k], v[2 * n + j] - v[2 * n + k]};
                        double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
                        for (int a = 0; a < 3; ++a) o[a] += h * w[a] + (hp / r) * dw * d[a];
                    }
                }
        out[k] = o[0];
        out[n + k] = o[1];
        out[2 * n + k] = o[2];
    }
}

/*
 * Short-range pair potential of each particle (Plummer-softened reading of the split):
 *   phi_SR,i = -Gm sum_{j in the 27 cells, 0 < r_ij < r_c} erfc(r_ij / (2 r_s)) / sqrt(r_ij^2 + eps^2)
 * (for eps = 0 the exact complement of the long-range potential -Gm erf(r/(2 r_s))/r).
 */
void sr_potential_cells(int64_t n, const double *pos, double box, int64_t n_c,
                        const int64_t *cell_of, const int64_t *order, const int64_t *cell_start,
                        double r_s, double r_c, double eps, double gm, double *phi)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
        int64_t c = cell_of[k];
        int64_t cx = c % n_c, cy = (c / n_c) % n_c, cz = c / (n_c * n_c);
        double s = 0.0;
        for (int64_t oz = -1; oz <= 1; ++oz)
            for (int64_t oy = -1; oy <= 1; ++oy)
                for (int64_t ox = -1; ox <= 1; ++ox) {
                    int64_t nc = ((((cz + oz + n_c) % n_c) * n_c + (cy + oy + n_c) % n_c) * n_c +
                                  (cx + ox + n_c) % n_c);
                    for (int64_t t = cell_start[nc]; t < cell_start[nc + 1]; ++t) {
                        int64_t j = order[t];
                        if (j == k) continue;
                        double dx = min_image(pos[j] - pos[k], box);
                        double dy = min_image(pos[n + j] - pos[n + k], box);
                        double dz = min_image(pos[2 * n + j] - pos[2 * n + k], box);
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (!(r2 < r_c * r_c) || r2 == 0.0) continue;
                        s += erfc(0.5 * sqrt(r2) / r_s) / sqrt(r2 + eps * eps);
                    }
                }
        phi[k] = -gm * s;
    }
}
