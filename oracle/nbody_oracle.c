/*
 * nbody_oracle.c -- plain FP64 CPU oracle for direct-summation gravity.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this file; only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark do.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes (Almerol et al., SC'25 workshops, Sec. 3, the force sum):
 *
 *     F_i = sum_{j != i} G m_i m_j (r_j - r_i) / r_ij^3
 *
 * divided by m_i (the paper computes the acceleration), with the Plummer
 * softening length eps inserted as r_ij^2 -> r_ij^2 + eps^2, plus the softened
 * potential at particle i due to all others:
 *
 *     a_i   =  G sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^(3/2)
 *     phi_i = -G sum_{j != i} m_j           / (|r_j - r_i|^2 + eps^2)^(1/2)
 *
 * Every quantity is IEEE double.  Each i runs one sequential j loop in
 * increasing j with Neumaier-compensated sums, so the result is the exact sum up
 * to one or two final roundings, and it does not depend on the OpenMP thread
 * count (threads only split the i loop).
 *
 * The time integrator is kick-drift-kick leapfrog (the paper says the
 * integration runs in FP64 on the host, Sec. 3, mixed-precision paragraph; it
 * does not name the scheme, KDK is the reading used here):
 *
 *     v_{1/2} = v + (dt/2) a(x);   x' = x + dt v_{1/2};   v' = v_{1/2} + (dt/2) a(x')
 *
 * Diagnostics: K = 1/2 sum m |v|^2, W = 1/2 sum m phi, E = K + W,
 * P = sum m v, L = sum m (x cross v).
 *
 * Jerk (the time derivative of the acceleration, which the paper computes
 * together with it, Sec. 3): with r = r_j - r_i, v = v_j - v_i, d2 = |r|^2 + eps^2,
 *
 *     jerk_i = G sum_{j != i} m_j [ v / d2^(3/2) - 3 (r . v) r / d2^(5/2) ]
 *
 * and the fourth-order Hermite predictor-corrector scheme that uses it
 * (Makino & Aarseth 1992), with one shared time step:
 *
 *     x_p = x + v dt + a dt^2/2 + j dt^3/6,   v_p = v + a dt + j dt^2/2
 *     a1, j1 <- forces and jerks at (x_p, v_p)
 *     v1 = v + (a + a1) dt/2 + (j - j1) dt^2/12
 *     x1 = x + (v + v1) dt/2 + (a - a1) dt^2/12
 *
 * Block (individual) time steps around the Hermite scheme -- the usual partner
 * of a jerk-based integrator in direct N-body codes (Makino & Aarseth 1992; the
 * paper does not describe its own stepping).  Every particle i carries its own
 * time t_i and a power-of-two step dt_i <= dt_max.  One block step:
 *   t_next = min_i (t_i + dt_i); the active set is {i : t_i + dt_i == t_next};
 *   every particle is predicted to t_next from its own (t_i, x, v, a, jerk);
 *   the active particles get a1, j1 from all predicted particles and are
 *   corrected over their own dt_i; their new step follows Aarseth's criterion
 *     dt_a = sqrt(eta (|a1| |a2| + |j1|^2) / (|j1| |a3| + |a2|^2))
 *   with a3 = (12 (a0 - a1) + 6 dt (j0 + j1)) / dt^3 and
 *        a2 = (-6 (a0 - a1) - dt (4 j0 + 2 j1)) / dt^2 + dt a3 (both at t_next),
 *   quantised: halve dt_i until dt_i <= dt_a (not below dt_min); double it
 *   when dt_a >= 2 dt_i, 2 dt_i <= dt_max and t_next is a multiple of 2 dt_i.
 * Initial steps: dt_i = the largest power of two <= min(dt_max, eta_s |a|/|j|),
 * not below dt_min.
 *
 * Layout: positions, velocities and accelerations are structure-of-arrays
 * [3][n] (x row, then y row, then z row), masses and potentials are [n].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Neumaier's improved Kahan summation: s + c carries the running sum. */
typedef struct {
    double s, c;
} csum;

static void csum_add(csum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double csum_get(const csum *a) { return a->s + a->c; }

/* Acceleration and potential on particle i from all j != i (the definition). */
static void oracle_one(int64_t n, const double *pos, const double *mass, double eps,
                       double G, int64_t i, double out[4]) {
    const double *x = pos, *y = pos + n, *z = pos + 2 * n;
    csum ax = {0, 0}, ay = {0, 0}, az = {0, 0}, ph = {0, 0};
    const double eps2 = eps * eps;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue; /* the sum excludes j = i */
        double dx = x[j] - x[i];
        double dy = y[j] - y[i];
        double dz = z[j] - z[i];
        double r2 = dx * dx + dy * dy + dz * dz + eps2;
        if (r2 == 0.0) continue; /* eps = 0 and coincident particles: no defined force */
        double r = sqrt(r2);
        double r3 = r2 * r; /* (r^2 + eps^2)^(3/2) */
        csum_add(&ax, mass[j] * dx / r3);
        csum_add(&ay, mass[j] * dy / r3);
        csum_add(&az, mass[j] * dz / r3);
        csum_add(&ph, mass[j] / r);
    }
    out[0] = G * csum_get(&ax);
    out[1] = G * csum_get(&ay);
    out[2] = G * csum_get(&az);
    out[3] = -G * csum_get(&ph);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* acc: [3][n] (may be NULL), pot: [n] (may be NULL). */
void oracle_forces(int64_t n, const double *pos, const double *mass, double eps, double G,
                   double *acc, double *pot) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double o[4];
        oracle_one(n, pos, mass, eps, G, i, o);
        if (acc) {
            acc[i] = o[0];
            acc[n + i] = o[1];
            acc[2 * n + i] = o[2];
        }
        if (pot) pot[i] = o[3];
    }
}

/* The same quantity for a subset of rows: acc is [3][nrows], pot is [nrows]. */
void oracle_forces_rows(int64_t n, const double *pos, const double *mass, double eps, double G,
                        const int64_t *rows, int64_t nrows, double *acc, double *pot) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nrows; ++k) {
        double o[4];
        oracle_one(n, pos, mass, eps, G, rows[k], o);
        if (acc) {
            acc[k] = o[0];
            acc[nrows + k] = o[1];
            acc[2 * nrows + k] = o[2];
        }
        if (pot) pot[k] = o[3];
    }
}

/* out[9] = K, W, E, Px, Py, Pz, Lx, Ly, Lz. */
void oracle_energy(int64_t n, const double *pos, const double *vel, const double *mass,
                   const double *pot, double *out) {
    csum k = {0, 0}, w = {0, 0}, p[3] = {{0, 0}, {0, 0}, {0, 0}}, l[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t i = 0; i < n; ++i) {
        double x = pos[i], y = pos[n + i], zz = pos[2 * n + i];
        double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i];
        double m = mass[i];
        csum_add(&k, 0.5 * m * (vx * vx + vy * vy + vz * vz));
        csum_add(&w, 0.5 * m * pot[i]);
        csum_add(&p[0], m * vx);
        csum_add(&p[1], m * vy);
        csum_add(&p[2], m * vz);
        csum_add(&l[0], m * (y * vz - zz * vy));
        csum_add(&l[1], m * (zz * vx - x * vz));
        csum_add(&l[2], m * (x * vy - y * vx));
    }
    out[0] = csum_get(&k);
    out[1] = csum_get(&w);
    out[2] = out[0] + out[1];
    for (int d = 0; d < 3; ++d) {
        out[3 + d] = csum_get(&p[d]);
        out[6 + d] = csum_get(&l[d]);
    }
}

/*
 * nsteps of KDK leapfrog, in place on pos and vel.
 * acc/pot: on entry the acceleration/potential at the initial positions if
 * have_acc != 0 (else they are computed first); on exit those at the final
 * positions.  diag (may be NULL): [nsteps + 1][9], row 0 the initial state and
 * row s the state after step s (oracle_energy layout).
 */
void oracle_kdk(int64_t n, double *pos, double *vel, const double *mass, double eps, double G,
                double dt, int64_t nsteps, double *acc, double *pot, int have_acc, double *diag) {
    if (!have_acc) oracle_forces(n, pos, mass, eps, G, acc, pot);
    if (diag) oracle_energy(n, pos, vel, mass, pot, diag);
    const double h = 0.5 * dt;
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t q = 0; q < 3 * n; ++q) vel[q] += h * acc[q]; /* kick */
        for (int64_t q = 0; q < 3 * n; ++q) pos[q] += dt * vel[q]; /* drift */
        oracle_forces(n, pos, mass, eps, G, acc, pot);
        for (int64_t q = 0; q < 3 * n; ++q) vel[q] += h * acc[q]; /* kick */
        if (diag) oracle_energy(n, pos, vel, mass, pot, diag + 9 * (s + 1));
    }
}

/* Acceleration, jerk and potential on particle i (the definitions above). */
static void oracle_one_jerk(int64_t n, const double *pos, const double *vel, const double *mass,
                            double eps, double G, int64_t i, double out[7]) {
    const double *x = pos, *y = pos + n, *z = pos + 2 * n;
    const double *vx = vel, *vy = vel + n, *vz = vel + 2 * n;
    csum s[7] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const double eps2 = eps * eps;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double rx = x[j] - x[i], ry = y[j] - y[i], rz = z[j] - z[i];
        double ux = vx[j] - vx[i], uy = vy[j] - vy[i], uz = vz[j] - vz[i];
        double d2 = rx * rx + ry * ry + rz * rz + eps2;
        if (d2 == 0.0) continue;
        double d = sqrt(d2);
        double d3 = d2 * d;      /* d2^(3/2) */
        double d5 = d3 * d2;     /* d2^(5/2) */
        double rv = rx * ux + ry * uy + rz * uz;
        csum_add(&s[0], mass[j] * rx / d3);
        csum_add(&s[1], mass[j] * ry / d3);
        csum_add(&s[2], mass[j] * rz / d3);
        csum_add(&s[3], mass[j] * (ux / d3 - 3.0 * rv * rx / d5));
        csum_add(&s[4], mass[j] * (uy / d3 - 3.0 * rv * ry / d5));
        csum_add(&s[5], mass[j] * (uz / d3 - 3.0 * rv * rz / d5));
        csum_add(&s[6], mass[j] / d);
    }
    for (int k = 0; k < 6; ++k) out[k] = G * csum_get(&s[k]);
    out[6] = -G * csum_get(&s[6]);
}

/* acc, jerk: [3][n]; pot: [n] (pot may be NULL). */
void oracle_forces_jerk(int64_t n, const double *pos, const double *vel, const double *mass,
                        double eps, double G, double *acc, double *jerk, double *pot) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double o[7];
        oracle_one_jerk(n, pos, vel, mass, eps, G, i, o);
        for (int d = 0; d < 3; ++d) {
            acc[d * n + i] = o[d];
            jerk[d * n + i] = o[3 + d];
        }
        if (pot) pot[i] = o[6];
    }
}

/* The same for rows[0..k): acc, jerk [3][k], pot [k] (sampled checks at large n). */
void oracle_forces_jerk_rows(int64_t n, const double *pos, const double *vel, const double *mass,
                             double eps, double G, const int64_t *rows, int64_t k, double *acc,
                             double *jerk, double *pot) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < k; ++r) {
        double o[7];
        oracle_one_jerk(n, pos, vel, mass, eps, G, rows[r], o);
        for (int d = 0; d < 3; ++d) {
            acc[d * k + r] = o[d];
            jerk[d * k + r] = o[3 + d];
        }
        pot[r] = o[6];
    }
}

/*
 * nsteps Hermite steps in place on pos and vel; acc/jerk/pot as in oracle_kdk
 * (computed first unless have != 0), diag as in oracle_kdk.
 */
void oracle_hermite(int64_t n, double *pos, double *vel, const double *mass, double eps, double G,
                    double dt, int64_t nsteps, double *acc, double *jerk, double *pot, int have,
                    double *diag) {
    if (!have) oracle_forces_jerk(n, pos, vel, mass, eps, G, acc, jerk, pot);
    if (diag) oracle_energy(n, pos, vel, mass, pot, diag);
    double *xp = malloc(sizeof(double) * 3 * n), *vp = malloc(sizeof(double) * 3 * n);
    double *a1 = malloc(sizeof(double) * 3 * n), *j1 = malloc(sizeof(double) * 3 * n);
    const double dt2 = dt * dt, dt3 = dt2 * dt;
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t q = 0; q < 3 * n; ++q) {  /* predictor */
            xp[q] = pos[q] + vel[q] * dt + acc[q] * dt2 / 2.0 + jerk[q] * dt3 / 6.0;
            vp[q] = vel[q] + acc[q] * dt + jerk[q] * dt2 / 2.0;
        }
        oracle_forces_jerk(n, xp, vp, mass, eps, G, a1, j1, pot);
        for (int64_t q = 0; q < 3 * n; ++q) {  /* corrector */
            double v1 = vel[q] + (acc[q] + a1[q]) * dt / 2.0 + (jerk[q] - j1[q]) * dt2 / 12.0;
            pos[q] = pos[q] + (vel[q] + v1) * dt / 2.0 + (acc[q] - a1[q]) * dt2 / 12.0;
            vel[q] = v1;
            acc[q] = a1[q];
            jerk[q] = j1[q];
        }
        if (diag) oracle_energy(n, pos, vel, mass, pot, diag + 9 * (s + 1));
    }
    free(xp);
    free(vp);
    free(a1);
    free(j1);
}

/* Acceleration, jerk and potential on particle i from all j, with every j taken
 * at the predicted state (xp, vp) and i at (xi, vi) -- the same definition as
 * oracle_one_jerk. */
static void oracle_one_jerk_at(int64_t n, const double *xp, const double *vp, const double *mass,
                               double eps, double G, int64_t i, double out[7]) {
    oracle_one_jerk(n, xp, vp, mass, eps, G, i, out);
}

static double norm3(const double *q, int64_t n, int64_t i) {
    double x = q[i], y = q[n + i], z = q[2 * n + i];
    return sqrt(x * x + y * y + z * z);
}

static double pow2_floor(double x) { return exp2(floor(log2(x))); }

/*
 * Aarseth's step criterion at the end of a Hermite step of length h (Makino &
 * Aarseth 1992): with a0, j0 the acceleration and jerk at the step start and
 * a1, j1 at its end, the cubic Hermite interpolant of a(t) gives the third
 * derivative a3 (constant over the step) and the second derivative at the step
 * start, which a3 carries to the step end:
 *   a3 = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3
 *   a2 = (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2 + h a3
 * and the criterion is sqrt(eta (|a1| |a2| + |j1|^2) / (|j1| |a3| + |a2|^2)),
 * or dt_max when the denominator vanishes.
 */
double oracle_aarseth_step(const double a0[3], const double j0[3], const double a1[3],
                           const double j1[3], double h, double eta, double dt_max) {
    double h2 = h * h, h3 = h2 * h;
    double a2[3], a3[3];
    for (int d = 0; d < 3; ++d) {
        a3[d] = (12.0 * (a0[d] - a1[d]) + 6.0 * h * (j0[d] + j1[d])) / h3;
        a2[d] = (-6.0 * (a0[d] - a1[d]) - h * (4.0 * j0[d] + 2.0 * j1[d])) / h2 + h * a3[d];
    }
    double na = sqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
    double nj = sqrt(j1[0] * j1[0] + j1[1] * j1[1] + j1[2] * j1[2]);
    double n2 = sqrt(a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]);
    double n3 = sqrt(a3[0] * a3[0] + a3[1] * a3[1] + a3[2] * a3[2]);
    double den = nj * n3 + n2 * n2;
    return den > 0.0 ? sqrt(eta * (na * n2 + nj * nj) / den) : dt_max;
}

/*
 * Block-step Hermite until every particle reaches t_end (a multiple of dt_max).
 * pos, vel in/out [3][n]; acc, jerk out [3][n] at t_end; pot out [n] at the
 * final predicted state of each particle's last step; dt_out [n] final steps;
 * returns the number of block steps, and the number of force evaluations of
 * single particles in *n_evals.  dt_max and dt_min are powers of two.
 */
int64_t oracle_block_hermite(int64_t n, double *pos, double *vel, const double *mass, double eps,
                             double G, double t_end, double dt_max, double dt_min, double eta,
                             double eta_s, double *acc, double *jerk, double *pot, double *dt_out,
                             int64_t *n_evals) {
    double *t = malloc(sizeof(double) * n), *dt = malloc(sizeof(double) * n);
    double *xp = malloc(sizeof(double) * 3 * n), *vp = malloc(sizeof(double) * 3 * n);
    oracle_forces_jerk(n, pos, vel, mass, eps, G, acc, jerk, pot);
    for (int64_t i = 0; i < n; ++i) {
        double an = norm3(acc, n, i), jn = norm3(jerk, n, i);
        double d = jn > 0.0 ? eta_s * an / jn : dt_max;
        if (!(d < dt_max)) d = dt_max;
        d = pow2_floor(d);
        if (d < dt_min) d = dt_min;
        t[i] = 0.0;
        dt[i] = d;
    }
    int64_t blocks = 0, evals = 0;
    for (;;) {
        double tn = INFINITY;
        for (int64_t i = 0; i < n; ++i)
            if (t[i] + dt[i] < tn) tn = t[i] + dt[i];
        if (n == 0 || tn > t_end) break;
        for (int64_t i = 0; i < n; ++i) { /* predict every particle to tn */
            double h = tn - t[i], h2 = h * h, h3 = h2 * h;
            for (int d = 0; d < 3; ++d) {
                int64_t q = d * n + i;
                xp[q] = pos[q] + vel[q] * h + acc[q] * h2 / 2.0 + jerk[q] * h3 / 6.0;
                vp[q] = vel[q] + acc[q] * h + jerk[q] * h2 / 2.0;
            }
        }
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            if (t[i] + dt[i] != tn) continue;
            double o[7];
            oracle_one_jerk_at(n, xp, vp, mass, eps, G, i, o);
            double h = dt[i], h2 = h * h;
            double a0[3], j0[3], a1[3], j1[3];
            for (int d = 0; d < 3; ++d) { /* corrector */
                int64_t q = d * n + i;
                a0[d] = acc[q];
                j0[d] = jerk[q];
                a1[d] = o[d];
                j1[d] = o[3 + d];
                double v1 = vel[q] + (acc[q] + a1[d]) * h / 2.0 + (jerk[q] - j1[d]) * h2 / 12.0;
                pos[q] = pos[q] + (vel[q] + v1) * h / 2.0 + (acc[q] - a1[d]) * h2 / 12.0;
                vel[q] = v1;
                acc[q] = a1[d];
                jerk[q] = j1[d];
            }
            pot[i] = o[6];
            /* next step: halve while above the criterion (not below dt_min),
             * or double once when the doubled step is allowed */
            double da = oracle_aarseth_step(a0, j0, a1, j1, h, eta, dt_max);
            double nd = h;
            while (nd > da && nd > dt_min) nd /= 2.0;
            if (nd == h && da >= 2.0 * h && 2.0 * h <= dt_max && fmod(tn, 2.0 * h) == 0.0) nd = 2.0 * h;
            t[i] = tn;
            dt[i] = nd;
        }
        for (int64_t i = 0; i < n; ++i)
            if (t[i] == tn) ++evals;
        ++blocks;
    }
    for (int64_t i = 0; i < n; ++i) dt_out[i] = dt[i];
    *n_evals = evals;
    free(t);
    free(dt);
    free(xp);
    free(vp);
    return blocks;
}
