/*
 * FP64 CPU oracle for the variable-speed-of-sound D2Q9 lattice Boltzmann model
 * (Buick & Cosgrove, "Investigation of a Lattice Boltzmann Model with a
 * Variable Speed of Sound").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the bench's CPU-baseline leg and the smoke check
 * do.  It shares no code, header, table or helper with the CUDA library.
 *
 * It is the update written out plainly, in the paper's order, in double
 * precision, with no blocking, fusion or reordering:
 *
 *   Section 2, Eq. 1 (bolt)  f_i(x+e_i,t+1) - f_i(x,t) = -(f_i - fbar_i)/tau
 *   Section 2, Eq. 2         fbar_i = w_i rho [1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u^2]
 *   Section 2, Eq. 3         rho = sum_i f_i ,  rho u = sum_i f_i e_i
 *   Section 2                w_0 = 4/9, w_1..4 = 1/9, w_5..8 = 1/36
 *   Section 2                e_i for i = 1..4 (axes) and i = 5..8 (diagonals)
 *   Section 3, Eq. 5 (nbm)   the same update plus the source 3 w_i alpha grad(rho).e_i
 *   Section 4                grad(rho) by central differences (the stable
 *                            choice); the forward difference the paper tried
 *                            first is kept as an option for the stability study.
 *
 * Readings taken where the paper is silent:
 *   - The state f_i(x,t) held here is the pre-collision distribution at time t
 *     (already streamed).  One step computes rho, u and grad(rho) at every site
 *     from that state first, then collides every site, then streams.
 *   - grad(rho) uses the same pre-collision rho as the equilibrium.
 *   - The central difference is the axis-aligned two-point stencil
 *     (rho(x+1)-rho(x-1))/2 in x and y; the forward difference is
 *     rho(x+1)-rho(x) in x and y.  Both wrap periodically.
 *   - The boundaries are periodic in x and y (the paper's wave runs of Section 4).
 *   - Moments are reported literally from Eq. 3, with no half-force shift.
 *
 * Arrays: f is [9][ny][nx] (direction-major, then row y, then column x);
 * fields rho, ux, uy and alpha are [ny][nx].
 *
 * Threads: the site loops carry an OpenMP "parallel for" when compiled with
 * -fopenmp.  It splits sites between threads only; each site's arithmetic is
 * the same as in the serial program, so the result does not depend on the
 * thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Link vectors e_i and weights w_i, Section 2. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                            1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

#define GRAD_CENTRAL 0
#define GRAD_FORWARD 1

static int wrap(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* Equilibrium distribution, Section 2, Eq. 2. */
void oracle_equilibrium(double rho, double ux, double uy, double *feq) {
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = W[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
    }
}

/* Density and velocity from the distributions at one site, Section 2, Eq. 3. */
static void site_moments(const double *fs, double *rho, double *ux, double *uy) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; i++) {
        r += fs[i];
        jx += fs[i] * EX[i];
        jy += fs[i] * EY[i];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* f_i(x,0) = fbar_i(rho(x), u(x)): the initial state is the local equilibrium
 * of the given fields (the paper gives only rho and u at t = 0). */
void oracle_init(int nx, int ny, const double *rho, const double *ux,
                 const double *uy, double *f) {
    long n = (long)nx * ny;
    for (long s = 0; s < n; s++) {
        double feq[9];
        oracle_equilibrium(rho[s], ux[s], uy[s], feq);
        for (int i = 0; i < 9; i++) f[i * n + s] = feq[i];
    }
}

/* rho, u at every site from the state f, Section 2, Eq. 3. */
void oracle_moments(int nx, int ny, const double *f, double *rho, double *ux,
                    double *uy) {
    long n = (long)nx * ny;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; s++) {
        double fs[9];
        for (int i = 0; i < 9; i++) fs[i] = f[i * n + s];
        site_moments(fs, &rho[s], &ux[s], &uy[s]);
    }
}

/* One time step of Section 3, Eq. 5, periodic in x and y.
 *   f      [9][ny][nx]  state at time t on entry, at t+1 on return
 *   work   [9][ny][nx]  scratch
 *   alpha  [ny][nx]     force amplitude per site (constant in the paper; a
 *                       field allows the spatially varying alpha of Section 5)
 *   rho,ux,uy [ny][nx]  scratch for the moments of the state at time t
 */
void oracle_step_field(int nx, int ny, double tau, const double *alpha,
                       int grad_mode, double *f, double *work, double *rho,
                       double *ux, double *uy) {
    long n = (long)nx * ny;

    /* 1. rho and u at every site (Eq. 3). */
    oracle_moments(nx, ny, f, rho, ux, uy);

    /* 2. Collide every site: BGK relaxation towards fbar (Eq. 2) plus the
     *    force 3 w_i alpha grad(rho).e_i (Eq. 5). */
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; s++) {
        int x = (int)(s % nx), y = (int)(s / nx);
        double gx, gy;
        if (grad_mode == GRAD_FORWARD) {
            gx = rho[(long)y * nx + wrap(x + 1, nx)] - rho[s];
            gy = rho[(long)wrap(y + 1, ny) * nx + x] - rho[s];
        } else {
            gx = 0.5 * (rho[(long)y * nx + wrap(x + 1, nx)] -
                        rho[(long)y * nx + wrap(x - 1, nx)]);
            gy = 0.5 * (rho[(long)wrap(y + 1, ny) * nx + x] -
                        rho[(long)wrap(y - 1, ny) * nx + x]);
        }
        double feq[9];
        oracle_equilibrium(rho[s], ux[s], uy[s], feq);
        for (int i = 0; i < 9; i++) {
            double fi = f[i * n + s];
            double force = 3.0 * W[i] * alpha[s] * (gx * EX[i] + gy * EY[i]);
            work[i * n + s] = fi - (fi - feq[i]) / tau + force;
        }
    }

    /* 3. Stream: the post-collision value at x moves to x + e_i (Eq. 5, left
     *    hand side), with periodic wrap. */
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; s++) {
        int x = (int)(s % nx), y = (int)(s / nx);
        for (int i = 0; i < 9; i++) {
            long d = (long)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
            f[i * n + d] = work[i * n + s];
        }
    }
}

/* One step of the driven channel of Section 4 (the runs of Fig. 1).  The
 * paper prescribes rho(t) and u = 0 at x = 0 and rho = 1, u = 0 at the far end
 * without giving a boundary scheme; the reading taken here is equilibrium
 * columns: after the collision, the post-collision distributions of column
 * x = 0 are replaced by fbar(rho_left, u = 0) and those of the last two
 * columns by fbar(rho_right, u = 0), then everything streams as usual.  The
 * far-end condition spans two columns so that the periodic wrap in x, which
 * brings column 0's values into column nx-1, reaches no interior gradient:
 * the density of column nx-1 enters only the gradients of columns nx-2 and 0,
 * both of which are overwritten.  Periodic in y.  Needs nx >= 4. */
void oracle_step_driven(int nx, int ny, double tau, const double *alpha, double rho_left,
                        double rho_right, double *f, double *work, double *rho, double *ux,
                        double *uy) {
    long n = (long)nx * ny;
    oracle_moments(nx, ny, f, rho, ux, uy);
    for (long s = 0; s < n; s++) {
        int x = (int)(s % nx), y = (int)(s / nx);
        double gx = 0.5 * (rho[(long)y * nx + wrap(x + 1, nx)] -
                           rho[(long)y * nx + wrap(x - 1, nx)]);
        double gy = 0.5 * (rho[(long)wrap(y + 1, ny) * nx + x] -
                           rho[(long)wrap(y - 1, ny) * nx + x]);
        double feq[9];
        oracle_equilibrium(rho[s], ux[s], uy[s], feq);
        for (int i = 0; i < 9; i++) {
            double fi = f[i * n + s];
            double force = 3.0 * W[i] * alpha[s] * (gx * EX[i] + gy * EY[i]);
            work[i * n + s] = fi - (fi - feq[i]) / tau + force;
        }
    }
    for (int y = 0; y < ny; y++) {
        double fl[9], fr[9];
        oracle_equilibrium(rho_left, 0.0, 0.0, fl);
        oracle_equilibrium(rho_right, 0.0, 0.0, fr);
        for (int i = 0; i < 9; i++) {
            work[i * n + (long)y * nx] = fl[i];
            work[i * n + (long)y * nx + nx - 2] = fr[i];
            work[i * n + (long)y * nx + nx - 1] = fr[i];
        }
    }
    for (long s = 0; s < n; s++) {
        int x = (int)(s % nx), y = (int)(s / nx);
        for (int i = 0; i < 9; i++) {
            long d = (long)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
            f[i * n + d] = work[i * n + s];
        }
    }
}

/* Runs `steps` driven-channel steps, the step from time t to t+1 using
 * rho_left(t) = 1 + amp sin(2 pi t / period) (Section 4: a sinusoidal density
 * with a period of 500 steps in the paper), rho_right = 1, for
 * t = t0 .. t0+steps-1; one alpha for the grid. */
int oracle_run_driven(int nx, int ny, double tau, double alpha, long t0, long steps, double amp,
                      double period, double *f) {
    long n = (long)nx * ny;
    if (nx < 4) return -2;
    double *work = (double *)malloc(sizeof(double) * 9 * n);
    double *buf = (double *)malloc(sizeof(double) * 4 * n);
    if (!work || !buf) {
        free(work);
        free(buf);
        return -1;
    }
    double *al = buf, *rho = buf + n, *ux = buf + 2 * n, *uy = buf + 3 * n;
    for (long s = 0; s < n; s++) al[s] = alpha;
    const double two_pi = 6.283185307179586476925287;
    for (long t = t0; t < t0 + steps; t++)
        oracle_step_driven(nx, ny, tau, al, 1.0 + amp * sin(two_pi * (double)t / period), 1.0, f,
                           work, rho, ux, uy);
    free(work);
    free(buf);
    return 0;
}

/* Runs `steps` steps with one alpha for the whole grid. */
int oracle_run(int nx, int ny, double tau, double alpha, int grad_mode,
               long steps, double *f) {
    long n = (long)nx * ny;
    double *work = (double *)malloc(sizeof(double) * 9 * n);
    double *buf = (double *)malloc(sizeof(double) * 4 * n);
    if (!work || !buf) {
        free(work);
        free(buf);
        return -1;
    }
    double *al = buf, *rho = buf + n, *ux = buf + 2 * n, *uy = buf + 3 * n;
    for (long s = 0; s < n; s++) al[s] = alpha;
    for (long t = 0; t < steps; t++)
        oracle_step_field(nx, ny, tau, al, grad_mode, f, work, rho, ux, uy);
    free(work);
    free(buf);
    return 0;
}

/* Runs `steps` steps with a per-site alpha field [ny][nx]. */
int oracle_run_field(int nx, int ny, double tau, const double *alpha,
                     int grad_mode, long steps, double *f) {
    long n = (long)nx * ny;
    double *work = (double *)malloc(sizeof(double) * 9 * n);
    double *buf = (double *)malloc(sizeof(double) * 3 * n);
    if (!work || !buf) {
        free(work);
        free(buf);
        return -1;
    }
    for (long t = 0; t < steps; t++)
        oracle_step_field(nx, ny, tau, alpha, grad_mode, f, work, buf, buf + n,
                          buf + 2 * n);
    free(work);
    free(buf);
    return 0;
}

/* Total mass sum_x rho and momentum sum_x rho u of the state (Eq. 3 summed
 * over the grid). */
void oracle_sums(int nx, int ny, const double *f, double *out3) {
    long n = (long)nx * ny;
    double m = 0.0, px = 0.0, py = 0.0;
    for (long s = 0; s < n; s++)
        for (int i = 0; i < 9; i++) {
            m += f[i * n + s];
            px += f[i * n + s] * EX[i];
            py += f[i * n + s] * EY[i];
        }
    out3[0] = m;
    out3[1] = px;
    out3[2] = py;
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Sets the number of OpenMP threads the site loops use (no effect without
 * OpenMP); returns the number that will be used. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
