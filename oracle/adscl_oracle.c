/*
 * adscl_oracle.c -- plain, sequential FP64 reference of the AdS4 Einstein-Klein-Gordon
 * method-of-lines scheme (Liebling & Khanna, arXiv:1706.07413, Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call this
 * file: only the tests, the package's smoke check and the CPU-baseline leg of the bench
 * use it.  It shares no code, header, table or constant generator with the CUDA library.
 *
 * Everything here is written for a reader checking it against the paper by eye: no
 * blocking, no fusion, no reordering.  Radial integrations run sequentially, exactly as
 * the paper describes the constraint solve (Sec. II, after Eq. (eq:delta)).
 *
 * Notation (Sec. II, Eq. (metric)): grid x_i = i h, i = 0..N-1, h = pi/(2(N-1));
 * rho = Phi^2 + Pi^2; s(x) = sin x cos x; F = A exp(-delta).
 *
 * Readings of the paper used here (the paper is silent on them; both implementations use
 * the same reading):
 *  - node-centred grid with x_0 = 0 and x_{N-1} = pi/2;
 *  - parity ghosts: Phi odd / Pi even at x = 0; Phi even / Pi odd at x = pi/2;
 *    f = F Pi follows Pi, g = F Phi follows Phi;
 *  - midpoint values by the 4-point Lagrange formula (-u_{i-1}+9u_i+9u_{i+1}-u_{i+2})/16;
 *  - delta: Simpson's rule per cell, summed from x = pi/2 inwards (Eq. (eq:delta), delta(pi/2)=0);
 *  - A: the Hamiltonian constraint Eq. (eq:aprime) rewritten for the mass function
 *    m = (1-A) sin x / cos^3 x, which obeys m' = tan^2 x rho - sin x cos x rho m, m(0)=0,
 *    integrated cell by cell outwards with classic RK4 (midpoint data interpolated);
 *  - RHS: Eqs. (eq:phi), (eq:pi) with 4th-order centred differences; Eq. (eq:pi) kept in the
 *    paper's form tan^{-2}(tan^2 g)'; Pi-dot at x=0 by L'Hopital (3 D g); boundary rows
 *    Phi-dot(0) = Phi-dot(pi/2) = Pi-dot(pi/2) = 0;
 *  - Kreiss-Oliger dissipation sigma/(64h) (u_{i-3}-6u_{i-2}+15u_{i-1}-20u_i+15u_{i+1}-6u_{i+2}+u_{i+3})
 *    on every non-boundary row (not in the paper);
 *  - classic RK4 in time with the constraint solve at every stage;
 *  - collapse: the first step after which min_i A < theta; t_c by linear interpolation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* instance status codes (same meaning as the library's per-instance status) */
enum { ORC_RUNNING = 0, ORC_DONE = 1, ORC_COLLAPSED = 2, ORC_NONFINITE = 3 };

/* ------------------------------------------------------------------ grid helpers */

static double grid_h(int N) { return 0.5 * ORC_PI / (double)(N - 1); }

/* value of u at index i in [-3, N+2], using the parity rule:
 * u_{-k} = p0 * u_k and u_{N-1+k} = p1 * u_{N-1-k}. */
static double with_ghost(const double *u, int N, int i, double p0, double p1)
{
    if (i < 0) return p0 * u[-i];
    if (i > N - 1) return p1 * u[2 * (N - 1) - i];
    return u[i];
}

/* ------------------------------------------------------------------ constraints */

/*
 * Solve the two constraints (Eqs. (eq:aprime) and (eq:delta)) on one time slice.
 * Inputs Phi, Pi (length N).  Outputs A, delta (length N); m (length N, optional);
 * *mass = m(pi/2) = integral of tan^2 x A rho dx (the paper's mass, Sec. II).
 */
void orc_constraints(int N, const double *Phi, const double *Pi, double *A, double *delta,
                     double *m_out, double *mass)
{
    const double h = grid_h(N);
    double *rho = (double *)malloc(sizeof(double) * N);
    double *rhom = (double *)malloc(sizeof(double) * N);
    double *m = (double *)malloc(sizeof(double) * N);
    int i, c;

    for (i = 0; i < N; ++i) rho[i] = Phi[i] * Phi[i] + Pi[i] * Pi[i];

    /* rho at cell midpoints x_{c+1/2} from interpolated Phi and Pi */
    for (c = 0; c < N - 1; ++c) {
        double phm = (-with_ghost(Phi, N, c - 1, -1.0, 1.0) + 9.0 * Phi[c] + 9.0 * Phi[c + 1]
                      - with_ghost(Phi, N, c + 2, -1.0, 1.0)) / 16.0;
        double pim = (-with_ghost(Pi, N, c - 1, 1.0, -1.0) + 9.0 * Pi[c] + 9.0 * Pi[c + 1]
                      - with_ghost(Pi, N, c + 2, 1.0, -1.0)) / 16.0;
        rhom[c] = phm * phm + pim * pim;
    }

    /* delta' = -sin x cos x rho, delta(pi/2) = 0: Simpson per cell, inward */
    delta[N - 1] = 0.0;
    for (c = N - 2; c >= 0; --c) {
        double x0 = c * h, xm = (c + 0.5) * h, x1 = (c + 1) * h;
        double s0 = sin(x0) * cos(x0), sm = sin(xm) * cos(xm), s1 = sin(x1) * cos(x1);
        delta[c] = delta[c + 1] + h / 6.0 * (s0 * rho[c] + 4.0 * sm * rhom[c] + s1 * rho[c + 1]);
    }

    /* m' = a - b m, a = tan^2 x rho, b = sin x cos x rho, m(0) = 0: RK4 per cell, outward */
    m[0] = 0.0;
    for (c = 0; c < N - 1; ++c) {
        double x0 = c * h, xm = (c + 0.5) * h, x1 = (c + 1) * h;
        double a0 = tan(x0) * tan(x0) * rho[c];
        double am = tan(xm) * tan(xm) * rhom[c];
        double a1 = (c + 1 == N - 1) ? 0.0 : tan(x1) * tan(x1) * rho[c + 1];
        double b0 = sin(x0) * cos(x0) * rho[c];
        double bm = sin(xm) * cos(xm) * rhom[c];
        double b1 = sin(x1) * cos(x1) * rho[c + 1];
        double y = m[c];
        double k1 = a0 - b0 * y;
        double k2 = am - bm * (y + 0.5 * h * k1);
        double k3 = am - bm * (y + 0.5 * h * k2);
        double k4 = a1 - b1 * (y + h * k3);
        m[c + 1] = y + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    }

    /* A = 1 - m cos^3 x / sin x, with A = 1 at both ends (Sec. II boundary conditions) */
    A[0] = 1.0;
    A[N - 1] = 1.0;
    for (i = 1; i < N - 1; ++i) {
        double x = i * h;
        A[i] = 1.0 - m[i] * cos(x) * cos(x) * cos(x) / sin(x);
    }
    if (mass) *mass = m[N - 1];
    if (m_out) memcpy(m_out, m, sizeof(double) * N);
    free(rho);
    free(rhom);
    free(m);
}

/* ------------------------------------------------------------------ right-hand side */

/* Kreiss-Oliger term at row i for field u with ghost parities p0, p1 */
static double ko_term(const double *u, int N, int i, double p0, double p1, double sigma, double h)
{
    double d6 = with_ghost(u, N, i - 3, p0, p1) - 6.0 * with_ghost(u, N, i - 2, p0, p1)
              + 15.0 * with_ghost(u, N, i - 1, p0, p1) - 20.0 * u[i]
              + 15.0 * with_ghost(u, N, i + 1, p0, p1) - 6.0 * with_ghost(u, N, i + 2, p0, p1)
              + with_ghost(u, N, i + 3, p0, p1);
    return sigma / (64.0 * h) * d6;
}

/* 4th-order centred first derivative at row i with ghost parities p0, p1 */
static double d1(const double *u, int N, int i, double p0, double p1, double h)
{
    return (with_ghost(u, N, i - 2, p0, p1) - 8.0 * with_ghost(u, N, i - 1, p0, p1)
            + 8.0 * with_ghost(u, N, i + 1, p0, p1) - with_ghost(u, N, i + 2, p0, p1)) / (12.0 * h);
}

/*
 * Time derivatives of Phi and Pi (Eqs. (eq:phi), (eq:pi)) given the constraint solution
 * A, delta on the same slice.  Eq. (eq:pi) is discretised in the form the paper writes it,
 * Pi-dot = tan^{-2} x (tan^2 x F Phi)': the 4th-order difference of u = tan^2 x g divided by
 * tan^2 x (the expanded form g' + 2g/(sin x cos x) is unstable at both ends of the grid).
 * u is odd about x = 0 and even about x = pi/2, where its finite limit is taken from the
 * even extrapolation u_{N-1} = (4 u_{N-2} - u_{N-3}) / 3.
 */
void orc_rhs(int N, double sigma, const double *Phi, const double *Pi, const double *A,
             const double *delta, double *dPhi, double *dPi)
{
    const double h = grid_h(N);
    double *f = (double *)malloc(sizeof(double) * N);
    double *g = (double *)malloc(sizeof(double) * N);
    double *u = (double *)malloc(sizeof(double) * N);
    int i;
    for (i = 0; i < N; ++i) {
        double F = A[i] * exp(-delta[i]);
        f[i] = F * Pi[i];
        g[i] = F * Phi[i];
    }
    for (i = 0; i < N - 1; ++i) u[i] = tan(i * h) * tan(i * h) * g[i];
    u[N - 1] = (4.0 * u[N - 2] - u[N - 3]) / 3.0;
    /* x = 0: Phi stays 0; Pi-dot = 3 (F Phi)'(0) (limit of Eq. (eq:pi)) */
    dPhi[0] = 0.0;
    dPi[0] = 3.0 * d1(g, N, 0, -1.0, 1.0, h) + ko_term(Pi, N, 0, 1.0, -1.0, sigma, h);
    for (i = 1; i < N - 1; ++i) {
        double x = i * h;
        dPhi[i] = d1(f, N, i, 1.0, -1.0, h) + ko_term(Phi, N, i, -1.0, 1.0, sigma, h);
        dPi[i] = d1(u, N, i, -1.0, 1.0, h) / (tan(x) * tan(x))
               + ko_term(Pi, N, i, 1.0, -1.0, sigma, h);
    }
    /* x = pi/2: Phi = Pi = 0 held fixed */
    dPhi[N - 1] = 0.0;
    dPi[N - 1] = 0.0;
    free(f);
    free(g);
    free(u);
}

/* ------------------------------------------------------------------ time stepping */

/*
 * One classic RK4 step of size dt (Sec. II: Runge-Kutta method of lines), constraints solved
 * at every stage.  Phi, Pi are updated in place.
 */
void orc_rk4_step(int N, double dt, double sigma, double *Phi, double *Pi)
{
    size_t bytes = sizeof(double) * N;
    double *A = (double *)malloc(bytes), *dl = (double *)malloc(bytes);
    double *sPhi = (double *)malloc(bytes), *sPi = (double *)malloc(bytes);
    double *kPhi = (double *)malloc(bytes), *kPi = (double *)malloc(bytes);
    double *aPhi = (double *)malloc(bytes), *aPi = (double *)malloc(bytes);
    const double cstage[4] = {0.0, 0.5, 0.5, 1.0};
    const double wstage[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    int i, st;
    memcpy(sPhi, Phi, bytes);
    memcpy(sPi, Pi, bytes);
    memcpy(aPhi, Phi, bytes);
    memcpy(aPi, Pi, bytes);
    for (st = 0; st < 4; ++st) {
        if (st > 0) {
            for (i = 0; i < N; ++i) {
                sPhi[i] = Phi[i] + cstage[st] * dt * kPhi[i];
                sPi[i] = Pi[i] + cstage[st] * dt * kPi[i];
            }
        }
        orc_constraints(N, sPhi, sPi, A, dl, NULL, NULL);
        orc_rhs(N, sigma, sPhi, sPi, A, dl, kPhi, kPi);
        for (i = 0; i < N; ++i) {
            aPhi[i] += wstage[st] * dt * kPhi[i];
            aPi[i] += wstage[st] * dt * kPi[i];
        }
    }
    memcpy(Phi, aPhi, bytes);
    memcpy(Pi, aPi, bytes);
    free(A); free(dl); free(sPhi); free(sPi); free(kPhi); free(kPi); free(aPhi); free(aPi);
}

static double min_of(const double *u, int N)
{
    double v = u[0];
    int i;
    for (i = 1; i < N; ++i)
        if (u[i] < v) v = u[i];
    return v;
}

/*
 * Evolve one instance from step index n0 (time n0*dt) by at most nsteps RK4 steps, stopping
 * early at collapse (Sec. II: the code stops when min A falls to a small threshold theta and
 * records that time) or at a non-finite slice.
 *
 *   minA_in    min A of the starting slice (pass NaN to have it recomputed here)
 *   out[0..6]  t_reached, t_collapse (+inf if none), mass at the last slice, min A at the last
 *              slice, steps taken, status (ORC_*), delta(0) at the last slice
 *   mass_hist, minA_hist  optional, length nsteps+1: values at every slice visited
 * Phi, Pi are updated in place; A, delta receive the constraint solution of the last slice.
 */
int orc_evolve(int N, double dt, long n0, long nsteps, double sigma, double theta, double minA_in,
               double *Phi, double *Pi, double *A, double *delta, double *out,
               double *mass_hist, double *minA_hist)
{
    double mass = 0.0, minA, t_c = INFINITY;
    long n;
    int status = ORC_DONE;
    orc_constraints(N, Phi, Pi, A, delta, NULL, &mass);
    minA = isnan(minA_in) ? min_of(A, N) : minA_in;
    if (mass_hist) mass_hist[0] = mass;
    if (minA_hist) minA_hist[0] = minA;
    for (n = 0; n < nsteps; ++n) {
        double minA_new;
        orc_rk4_step(N, dt, sigma, Phi, Pi);
        orc_constraints(N, Phi, Pi, A, delta, NULL, &mass);
        minA_new = min_of(A, N);
        if (mass_hist) mass_hist[n + 1] = mass;
        if (minA_hist) minA_hist[n + 1] = minA_new;
        if (!isfinite(mass) || !isfinite(delta[0]) || !isfinite(minA_new)) {
            status = ORC_NONFINITE;
            minA = minA_new;
            ++n;
            break;
        }
        if (minA_new < theta) {
            /* linear interpolation of min A between t_n and t_{n+1} */
            double tn = (double)(n0 + n) * dt;
            t_c = tn + dt * (minA - theta) / (minA - minA_new);
            status = ORC_COLLAPSED;
            minA = minA_new;
            ++n;
            break;
        }
        minA = minA_new;
    }
    out[0] = (double)(n0 + n) * dt;
    out[1] = t_c;
    out[2] = mass;
    out[3] = minA;
    out[4] = (double)n;
    out[5] = (double)status;
    out[6] = delta[0];
    return status;
}

/* ==================================================================================== */
/* The paper's production variant (Sec. II): A is evolved with Eq. (eq:adot) instead of  */
/* being integrated from Eq. (eq:aprime) at every stage, and re-integrated from          */
/* Eq. (eq:aprime) only periodically; delta is still integrated at every stage; the time */
/* integrator is a Runge-Kutta method of second or third order (the paper's runs use     */
/* third order).  Readings: the strong-stability-preserving Runge-Kutta methods of       */
/* Shu and Osher (order 2: Heun's method; order 3: the three-stage SSP scheme), no       */
/* dissipation on A, A = 1 at both ends, and the mass by the composite Simpson rule of   */
/* M = int tan^2 x A rho dx on the nodes.                                                 */
/* ==================================================================================== */

/* A-dot of Eq. (eq:adot): -2 sin x cos x A^2 e^{-delta} Phi Pi; zero at both ends */
void orc_adot(int N, const double *Phi, const double *Pi, const double *A, const double *delta,
              double *dA)
{
    const double h = grid_h(N);
    int i;
    dA[0] = 0.0;
    dA[N - 1] = 0.0;
    for (i = 1; i < N - 1; ++i) {
        double x = i * h;
        dA[i] = -2.0 * sin(x) * cos(x) * A[i] * A[i] * exp(-delta[i]) * Phi[i] * Pi[i];
    }
}

/* M = int_0^{pi/2} tan^2 x A (Phi^2 + Pi^2) dx (Sec. II) by the composite Simpson rule on the
 * nodes (N - 1 is even); the integrand vanishes at x = 0 and tends to 0 at x = pi/2 */
double orc_mass_simpson(int N, const double *Phi, const double *Pi, const double *A)
{
    const double h = grid_h(N);
    double sum = 0.0;
    int i;
    for (i = 1; i < N - 1; ++i) {
        double x = i * h;
        double w = (i % 2 == 1) ? 4.0 : 2.0;
        sum += w * tan(x) * tan(x) * A[i] * (Phi[i] * Phi[i] + Pi[i] * Pi[i]);
    }
    return h / 3.0 * sum;
}

/* right-hand side L(Phi, Pi, A) of the evolved-A scheme: delta from the slice's Phi, Pi
 * (Eq. (eq:delta)), Phi-dot and Pi-dot as in orc_rhs with the slice's own A, A-dot by
 * Eq. (eq:adot) */
static void ea_rhs(int N, double sigma, const double *Phi, const double *Pi, const double *A,
                   double *dPhi, double *dPi, double *dA)
{
    size_t bytes = sizeof(double) * N;
    double *Ac = (double *)malloc(bytes), *dl = (double *)malloc(bytes);
    orc_constraints(N, Phi, Pi, Ac, dl, NULL, NULL);   /* only delta is used */
    orc_rhs(N, sigma, Phi, Pi, A, dl, dPhi, dPi);
    orc_adot(N, Phi, Pi, A, dl, dA);
    free(Ac);
    free(dl);
}

/*
 * One step of the evolved-A scheme with the Shu-Osher SSP Runge-Kutta method of order 2 or 3:
 *   order 2:  y1 = y + dt L(y);  y_new = y/2 + (y1 + dt L(y1))/2
 *   order 3:  y1 = y + dt L(y);  y2 = 3y/4 + (y1 + dt L(y1))/4;  y_new = y/3 + 2(y2 + dt L(y2))/3
 * y = (Phi, Pi, A), updated in place.
 */
void orc_ea_step(int N, int order, double dt, double sigma, double *Phi, double *Pi, double *A)
{
    size_t bytes = sizeof(double) * N;
    double *sP = (double *)malloc(bytes), *sQ = (double *)malloc(bytes), *sA = (double *)malloc(bytes);
    double *kP = (double *)malloc(bytes), *kQ = (double *)malloc(bytes), *kA = (double *)malloc(bytes);
    /* y^{(s+1)} = a_s y_n + b_s (y^{(s)} + dt L(y^{(s)})) */
    const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
    const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
    const double *a = (order == 2) ? a2 : a3, *b = (order == 2) ? b2 : b3;
    int st, i;
    memcpy(sP, Phi, bytes);
    memcpy(sQ, Pi, bytes);
    memcpy(sA, A, bytes);
    for (st = 0; st < order; ++st) {
        ea_rhs(N, sigma, sP, sQ, sA, kP, kQ, kA);
        for (i = 0; i < N; ++i) {
            sP[i] = a[st] * Phi[i] + b[st] * (sP[i] + dt * kP[i]);
            sQ[i] = a[st] * Pi[i] + b[st] * (sQ[i] + dt * kQ[i]);
            sA[i] = a[st] * A[i] + b[st] * (sA[i] + dt * kA[i]);
        }
    }
    memcpy(Phi, sP, bytes);
    memcpy(Pi, sQ, bytes);
    memcpy(A, sA, bytes);
    free(sP); free(sQ); free(sA); free(kP); free(kQ); free(kA);
}

/*
 * The fixed-metric case of the paper's Table II: A = 1 and delta = 0 held fixed, so that
 * Eqs. (eq:phi), (eq:pi) are the linear wave equation on AdS4.  One Shu-Osher SSP step of
 * order 2 or 3 of (Phi, Pi) with the same right-hand side and dissipation as orc_rhs.
 */
void orc_fixed_step(int N, int order, double dt, double sigma, double *Phi, double *Pi)
{
    size_t bytes = sizeof(double) * N;
    double *sP = (double *)malloc(bytes), *sQ = (double *)malloc(bytes);
    double *kP = (double *)malloc(bytes), *kQ = (double *)malloc(bytes);
    double *one = (double *)malloc(bytes), *zero = (double *)malloc(bytes);
    const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
    const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
    const double *a = (order == 2) ? a2 : a3, *b = (order == 2) ? b2 : b3;
    int st, i;
    for (i = 0; i < N; ++i) {
        one[i] = 1.0;
        zero[i] = 0.0;
    }
    memcpy(sP, Phi, bytes);
    memcpy(sQ, Pi, bytes);
    for (st = 0; st < order; ++st) {
        orc_rhs(N, sigma, sP, sQ, one, zero, kP, kQ);
        for (i = 0; i < N; ++i) {
            sP[i] = a[st] * Phi[i] + b[st] * (sP[i] + dt * kP[i]);
            sQ[i] = a[st] * Pi[i] + b[st] * (sQ[i] + dt * kQ[i]);
        }
    }
    memcpy(Phi, sP, bytes);
    memcpy(Pi, sQ, bytes);
    free(sP); free(sQ); free(kP); free(kQ); free(one); free(zero);
}

/*
 * Evolve one instance with the evolved-A scheme from step index n0 by at most nsteps steps.
 * The slice at step index n has A re-integrated from Eq. (eq:aprime) when reint > 0 and
 * n % reint == 0 (A is given as state otherwise).  Diagnostics of a slice: min A of its A,
 * the Simpson mass, delta(0).  Collapse and the outputs as in orc_evolve (out[2] = Simpson
 * mass).  Phi, Pi, A are the state (updated in place); delta receives the last slice's delta.
 */
int orc_ea_evolve(int N, int order, int reint, double dt, long n0, long nsteps, double sigma,
                  double theta, double minA_in, double *Phi, double *Pi, double *A, double *delta,
                  double *out)
{
    size_t bytes = sizeof(double) * N;
    double *Ac = (double *)malloc(bytes);
    double mass, minA, t_c = INFINITY;
    long n;
    int status = ORC_DONE;
    orc_constraints(N, Phi, Pi, Ac, delta, NULL, NULL);
    if (reint > 0 && n0 % reint == 0) memcpy(A, Ac, bytes);
    mass = orc_mass_simpson(N, Phi, Pi, A);
    minA = isnan(minA_in) ? min_of(A, N) : minA_in;
    for (n = 0; n < nsteps; ++n) {
        double minA_new;
        orc_ea_step(N, order, dt, sigma, Phi, Pi, A);
        orc_constraints(N, Phi, Pi, Ac, delta, NULL, NULL);
        if (reint > 0 && (n0 + n + 1) % reint == 0) memcpy(A, Ac, bytes);
        mass = orc_mass_simpson(N, Phi, Pi, A);
        minA_new = min_of(A, N);
        if (!isfinite(mass) || !isfinite(delta[0]) || !isfinite(minA_new)) {
            status = ORC_NONFINITE;
            minA = minA_new;
            ++n;
            break;
        }
        if (minA_new < theta) {
            double tn = (double)(n0 + n) * dt;
            t_c = tn + dt * (minA - theta) / (minA - minA_new);
            status = ORC_COLLAPSED;
            minA = minA_new;
            ++n;
            break;
        }
        minA = minA_new;
    }
    out[0] = (double)(n0 + n) * dt;
    out[1] = t_c;
    out[2] = mass;
    out[3] = minA;
    out[4] = (double)n;
    out[5] = (double)status;
    out[6] = delta[0];
    free(Ac);
    return status;
}

/* ------------------------------------------------------------------ AdS eigenbasis */

/* Jacobi polynomial P_n^{(a,b)}(y) by the standard three-term recurrence in n */
static double jacobi_p(int n, double a, double b, double y)
{
    double p0 = 1.0, p1, p2;
    int k;
    if (n == 0) return p0;
    p1 = 0.5 * ((a + b + 2.0) * y + (a - b));
    for (k = 2; k <= n; ++k) {
        double c = 2.0 * k + a + b;
        double lhs = 2.0 * k * (k + a + b) * (c - 2.0);
        double r1 = (c - 1.0) * (c * (c - 2.0) * y + a * a - b * b);
        double r2 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
        p2 = (r1 * p1 - r2 * p0) / lhs;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/*
 * Linear normal modes of the scalar on AdS4 (the spectrum of Sec. II; the paper gives no
 * formula, this is the standard result of the works it cites):
 *   e_j(x) = d_j cos^3 x P_j^{(1/2,3/2)}(cos 2x),  omega_j = 3 + 2j,
 *   d_j = 2 sqrt(j! (j+2)!) / Gamma(j + 3/2),  so that  int_0^{pi/2} e_i e_j tan^2 x dx = delta_ij.
 * Derivative via dP_n^{(a,b)}/dy = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}.
 * Outputs e[j*nx + i], de[j*nx + i] at the points x[i].
 */
void orc_eigen_at(int J, int nx, const double *x, double *e, double *de)
{
    int j, i;
    for (j = 0; j < J; ++j) {
        double dj = 2.0 * exp(0.5 * (lgamma(j + 1.0) + lgamma(j + 3.0)) - lgamma(j + 1.5));
        for (i = 0; i < nx; ++i) {
            double c = cos(x[i]), s = sin(x[i]), y = cos(2.0 * x[i]);
            double P = jacobi_p(j, 0.5, 1.5, y);
            double dP = (j == 0) ? 0.0 : 0.5 * (j + 3.0) * jacobi_p(j - 1, 1.5, 2.5, y);
            e[(size_t)j * nx + i] = dj * c * c * c * P;
            /* d/dx [cos^3 x P(cos 2x)] = -3 cos^2 x sin x P - 2 sin 2x cos^3 x P'(y) */
            de[(size_t)j * nx + i] = dj * (-3.0 * c * c * s * P - 4.0 * s * c * c * c * c * dP);
        }
    }
}

/* the same on the evolution grid x_i = i h */
void orc_eigen(int N, int J, double *e, double *de)
{
    double *x = (double *)malloc(sizeof(double) * N);
    const double h = grid_h(N);
    int i;
    for (i = 0; i < N; ++i) x[i] = i * h;
    orc_eigen_at(J, N, x, e, de);
    free(x);
}

/*
 * Mode energies: Pi_j = (sqrt(A) Pi, e_j), Phi_j = (sqrt(A) Phi, e_j'),
 * E_j = Pi_j^2 + Phi_j^2 / omega_j^2, with (u, v) = int_0^{pi/2} u v tan^2 x dx by the
 * trapezoid rule on the grid (the integrand vanishes at both ends).
 * Also returns the projections themselves if Pij/Phij are non-NULL.
 */
void orc_spectrum(int N, int J, const double *Phi, const double *Pi, const double *A, double *E,
                  double *Pij, double *Phij)
{
    const double h = grid_h(N);
    double *e = (double *)malloc(sizeof(double) * (size_t)N * J);
    double *de = (double *)malloc(sizeof(double) * (size_t)N * J);
    int j, i;
    orc_eigen(N, J, e, de);
    for (j = 0; j < J; ++j) {
        double pj = 0.0, fj = 0.0, om = 3.0 + 2.0 * j;
        for (i = 1; i < N - 1; ++i) {
            double x = i * h, t2 = tan(x) * tan(x), sa = sqrt(A[i]);
            pj += h * t2 * sa * Pi[i] * e[(size_t)j * N + i];
            fj += h * t2 * sa * Phi[i] * de[(size_t)j * N + i];
        }
        E[j] = pj * pj + fj * fj / (om * om);
        if (Pij) Pij[j] = pj;
        if (Phij) Phij[j] = fj;
    }
    free(e);
    free(de);
}

/*
 * Two of the three quantities that the two-time-framework (TTF) equations conserve (Sec. II:
 * the normal-mode decomposition connects the evolution with perturbation theory and its three
 * conserved quantities), written out from the mode energies of one slice:
 *   total energy      E = sum_{j<J} E_j,
 *   particle number   N = sum_{j<J} E_j / omega_j,   omega_j = 3 + 2j,
 * and the temperature T = E / N, the quantity the paper quotes for its quasi-periodic initial
 * data (it depends only on how the energy is distributed over the modes).  E_j is the energy of
 * mode j, so E_j / omega_j is its number of quanta.  The third conserved quantity, the TTF
 * Hamiltonian, needs the interaction coefficients of the resonant system, which the paper does
 * not give; it is not computed.  out[0..2] = E, N, T.
 */
void orc_ttf(int J, const double *E, double *out)
{
    double e_tot = 0.0, n_tot = 0.0;
    int j;
    for (j = 0; j < J; ++j) {
        e_tot += E[j];
        n_tot += E[j] / (3.0 + 2.0 * j);
    }
    out[0] = e_tot;
    out[1] = n_tot;
    out[2] = e_tot / n_tot;
}

/* Pi(x,0) = sum_j a_j e_j(x), Phi(x,0) = 0, with the boundary values of Sec. II imposed */
void orc_synthesize(int N, int K, const double *a, double *Phi, double *Pi)
{
    double *e = (double *)malloc(sizeof(double) * (size_t)N * K);
    double *de = (double *)malloc(sizeof(double) * (size_t)N * K);
    int j, i;
    orc_eigen(N, K, e, de);
    for (i = 0; i < N; ++i) {
        double v = 0.0;
        for (j = 0; j < K; ++j) v += a[j] * e[(size_t)j * N + i];
        Pi[i] = v;
        Phi[i] = 0.0;
    }
    Pi[N - 1] = 0.0;
    free(e);
    free(de);
}

/* ==================================================================================== */
/* Discrete adjoint (reverse mode) of the scheme above.  Every routine below transposes */
/* the corresponding forward routine line by line: given the sensitivity of a scalar    */
/* functional to the outputs, it accumulates (+=) the sensitivity to the inputs.        */
/* ==================================================================================== */

/* w_bar[mirror(j)] += p * val for a stencil entry that read with_ghost(w, N, j, p0, p1) */
static void scatter_ghost(double *wbar, int N, int j, double p0, double p1, double val)
{
    if (j < 0) wbar[-j] += p0 * val;
    else if (j > N - 1) wbar[2 * (N - 1) - j] += p1 * val;
    else wbar[j] += val;
}

/*
 * Transpose of orc_constraints: given Abar (length N) and dbar (length N), the sensitivities
 * to A and delta, accumulate the sensitivities to Phi and Pi.  A_0, A_{N-1} and delta_{N-1}
 * are constants and their bars are ignored.
 */
void orc_constraints_vjp(int N, const double *Phi, const double *Pi, const double *Abar,
                         const double *dbar_in, double *Phibar, double *Pibar)
{
    const double h = grid_h(N);
    double *rho = (double *)calloc(N, sizeof(double)), *rhom = (double *)calloc(N, sizeof(double));
    double *phm = (double *)calloc(N, sizeof(double)), *pim = (double *)calloc(N, sizeof(double));
    double *m = (double *)calloc(N, sizeof(double)), *mbar = (double *)calloc(N, sizeof(double));
    double *rhobar = (double *)calloc(N, sizeof(double)), *rhombar = (double *)calloc(N, sizeof(double));
    double *dbar = (double *)calloc(N, sizeof(double));
    int i, c;

    /* forward values needed by the transpose */
    for (i = 0; i < N; ++i) rho[i] = Phi[i] * Phi[i] + Pi[i] * Pi[i];
    for (c = 0; c < N - 1; ++c) {
        phm[c] = (-with_ghost(Phi, N, c - 1, -1.0, 1.0) + 9.0 * Phi[c] + 9.0 * Phi[c + 1]
                  - with_ghost(Phi, N, c + 2, -1.0, 1.0)) / 16.0;
        pim[c] = (-with_ghost(Pi, N, c - 1, 1.0, -1.0) + 9.0 * Pi[c] + 9.0 * Pi[c + 1]
                  - with_ghost(Pi, N, c + 2, 1.0, -1.0)) / 16.0;
        rhom[c] = phm[c] * phm[c] + pim[c] * pim[c];
    }
    m[0] = 0.0;
    for (c = 0; c < N - 1; ++c) {
        double x0 = c * h, xm = (c + 0.5) * h, x1 = (c + 1) * h;
        double a0 = tan(x0) * tan(x0) * rho[c], am = tan(xm) * tan(xm) * rhom[c];
        double a1 = (c + 1 == N - 1) ? 0.0 : tan(x1) * tan(x1) * rho[c + 1];
        double b0 = sin(x0) * cos(x0) * rho[c], bm = sin(xm) * cos(xm) * rhom[c];
        double b1 = sin(x1) * cos(x1) * rho[c + 1];
        double y = m[c];
        double k1 = a0 - b0 * y;
        double k2 = am - bm * (y + 0.5 * h * k1);
        double k3 = am - bm * (y + 0.5 * h * k2);
        double k4 = a1 - b1 * (y + h * k3);
        m[c + 1] = y + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    }

    /* A_i = 1 - m_i cos^3 x_i / sin x_i */
    for (i = 1; i < N - 1; ++i) {
        double x = i * h;
        mbar[i] += -Abar[i] * cos(x) * cos(x) * cos(x) / sin(x);
    }
    /* the outward RK4 recurrence for m, transposed (cells in reverse order) */
    for (c = N - 2; c >= 0; --c) {
        double x0 = c * h, xm = (c + 0.5) * h, x1 = (c + 1) * h;
        double t0 = tan(x0) * tan(x0), tm = tan(xm) * tan(xm), t1 = tan(x1) * tan(x1);
        double s0 = sin(x0) * cos(x0), sm = sin(xm) * cos(xm), s1 = sin(x1) * cos(x1);
        double a0 = t0 * rho[c], am = tm * rhom[c], a1 = (c + 1 == N - 1) ? 0.0 : t1 * rho[c + 1];
        double b0 = s0 * rho[c], bm = sm * rhom[c], b1 = s1 * rho[c + 1];
        double y = m[c];
        double k1 = a0 - b0 * y;
        double k2 = am - bm * (y + 0.5 * h * k1);
        double k3 = am - bm * (y + 0.5 * h * k2);
        double mb = mbar[c + 1];
        double yb = mb, k1b = h / 6.0 * mb, k2b = h / 3.0 * mb, k3b = h / 3.0 * mb, k4b = h / 6.0 * mb;
        double a0b = 0, amb = 0, a1b = 0, b0b = 0, bmb = 0, b1b = 0;
        /* k4 = a1 - b1 (y + h k3) */
        a1b += k4b;
        b1b -= k4b * (y + h * k3);
        yb -= k4b * b1;
        k3b -= k4b * b1 * h;
        /* k3 = am - bm (y + h/2 k2) */
        amb += k3b;
        bmb -= k3b * (y + 0.5 * h * k2);
        yb -= k3b * bm;
        k2b -= k3b * bm * 0.5 * h;
        /* k2 = am - bm (y + h/2 k1) */
        amb += k2b;
        bmb -= k2b * (y + 0.5 * h * k1);
        yb -= k2b * bm;
        k1b -= k2b * bm * 0.5 * h;
        /* k1 = a0 - b0 y */
        a0b += k1b;
        b0b -= k1b * y;
        yb -= k1b * b0;
        mbar[c] += yb;
        rhobar[c] += t0 * a0b + s0 * b0b;
        rhombar[c] += tm * amb + sm * bmb;
        if (c + 1 != N - 1) rhobar[c + 1] += t1 * a1b;
        rhobar[c + 1] += s1 * b1b;
    }
    /* delta_c = delta_{c+1} + h/6 (s0 rho_c + 4 sm rhom_c + s1 rho_{c+1}), transposed */
    for (i = 0; i < N; ++i) dbar[i] = dbar_in[i];
    dbar[N - 1] = 0.0;
    for (c = 0; c < N - 1; ++c) {
        double x0 = c * h, xm = (c + 0.5) * h, x1 = (c + 1) * h;
        double s0 = sin(x0) * cos(x0), sm = sin(xm) * cos(xm), s1 = sin(x1) * cos(x1);
        double db = dbar[c];
        if (c + 1 < N - 1) dbar[c + 1] += db;
        rhobar[c] += h / 6.0 * s0 * db;
        rhombar[c] += h / 6.0 * 4.0 * sm * db;
        rhobar[c + 1] += h / 6.0 * s1 * db;
    }
    /* rho at midpoints from the interpolated fields */
    for (c = 0; c < N - 1; ++c) {
        double pb = 2.0 * phm[c] * rhombar[c] / 16.0, qb = 2.0 * pim[c] * rhombar[c] / 16.0;
        scatter_ghost(Phibar, N, c - 1, -1.0, 1.0, -pb);
        Phibar[c] += 9.0 * pb;
        Phibar[c + 1] += 9.0 * pb;
        scatter_ghost(Phibar, N, c + 2, -1.0, 1.0, -pb);
        scatter_ghost(Pibar, N, c - 1, 1.0, -1.0, -qb);
        Pibar[c] += 9.0 * qb;
        Pibar[c + 1] += 9.0 * qb;
        scatter_ghost(Pibar, N, c + 2, 1.0, -1.0, -qb);
    }
    for (i = 0; i < N; ++i) {
        Phibar[i] += 2.0 * Phi[i] * rhobar[i];
        Pibar[i] += 2.0 * Pi[i] * rhobar[i];
    }
    free(rho); free(rhom); free(phm); free(pim); free(m); free(mbar); free(rhobar); free(rhombar);
    free(dbar);
}

/* transposed stencils: scatter val * (KO stencil at row i) and val * (D stencil at row i) */
static void ko_term_vjp(double *wbar, int N, int i, double p0, double p1, double sigma, double h, double val)
{
    double s = sigma / (64.0 * h) * val;
    scatter_ghost(wbar, N, i - 3, p0, p1, s);
    scatter_ghost(wbar, N, i - 2, p0, p1, -6.0 * s);
    scatter_ghost(wbar, N, i - 1, p0, p1, 15.0 * s);
    wbar[i] += -20.0 * s;
    scatter_ghost(wbar, N, i + 1, p0, p1, 15.0 * s);
    scatter_ghost(wbar, N, i + 2, p0, p1, -6.0 * s);
    scatter_ghost(wbar, N, i + 3, p0, p1, s);
}

static void d1_vjp(double *wbar, int N, int i, double p0, double p1, double h, double val)
{
    double s = val / (12.0 * h);
    scatter_ghost(wbar, N, i - 2, p0, p1, s);
    scatter_ghost(wbar, N, i - 1, p0, p1, -8.0 * s);
    scatter_ghost(wbar, N, i + 1, p0, p1, 8.0 * s);
    scatter_ghost(wbar, N, i + 2, p0, p1, -s);
}

/*
 * Transpose of orc_rhs: given vP, vQ (sensitivities to dPhi/dt, dPi/dt), accumulate the
 * sensitivities to Phi, Pi, A and delta.
 */
void orc_rhs_vjp(int N, double sigma, const double *Phi, const double *Pi, const double *A,
                 const double *delta, const double *vP, const double *vQ, double *Phibar,
                 double *Pibar, double *Abar, double *dbar)
{
    const double h = grid_h(N);
    double *F = (double *)calloc(N, sizeof(double));
    double *fb = (double *)calloc(N, sizeof(double)), *gb = (double *)calloc(N, sizeof(double));
    double *ub = (double *)calloc(N, sizeof(double));
    int i;
    for (i = 0; i < N; ++i) F[i] = A[i] * exp(-delta[i]);
    /* row 0: dPi = 3 d1(g, 0) + KO(Pi, 0) */
    d1_vjp(gb, N, 0, -1.0, 1.0, h, 3.0 * vQ[0]);
    ko_term_vjp(Pibar, N, 0, 1.0, -1.0, sigma, h, vQ[0]);
    for (i = 1; i < N - 1; ++i) {
        double x = i * h;
        d1_vjp(fb, N, i, 1.0, -1.0, h, vP[i]);
        ko_term_vjp(Phibar, N, i, -1.0, 1.0, sigma, h, vP[i]);
        d1_vjp(ub, N, i, -1.0, 1.0, h, vQ[i] / (tan(x) * tan(x)));
        ko_term_vjp(Pibar, N, i, 1.0, -1.0, sigma, h, vQ[i]);
    }
    /* u_{N-1} = (4 u_{N-2} - u_{N-3}) / 3 */
    ub[N - 2] += 4.0 / 3.0 * ub[N - 1];
    ub[N - 3] += -1.0 / 3.0 * ub[N - 1];
    ub[N - 1] = 0.0;
    for (i = 0; i < N - 1; ++i) gb[i] += tan(i * h) * tan(i * h) * ub[i];
    for (i = 0; i < N; ++i) {
        double Fb = fb[i] * Pi[i] + gb[i] * Phi[i];
        Pibar[i] += fb[i] * F[i];
        Phibar[i] += gb[i] * F[i];
        Abar[i] += Fb * exp(-delta[i]);
        dbar[i] += -Fb * F[i];
    }
    free(F); free(fb); free(gb); free(ub);
}

/* transpose of the full right-hand side R(y) = rhs(y, constraints(y)) */
static void rhs_full_vjp(int N, double sigma, const double *Phi, const double *Pi, const double *vP,
                         const double *vQ, double *Phibar, double *Pibar)
{
    size_t bytes = sizeof(double) * N;
    double *A = (double *)malloc(bytes), *dl = (double *)malloc(bytes);
    double *Ab = (double *)calloc(N, sizeof(double)), *db = (double *)calloc(N, sizeof(double));
    orc_constraints(N, Phi, Pi, A, dl, NULL, NULL);
    orc_rhs_vjp(N, sigma, Phi, Pi, A, dl, vP, vQ, Phibar, Pibar, Ab, db);
    orc_constraints_vjp(N, Phi, Pi, Ab, db, Phibar, Pibar);
    free(A); free(dl); free(Ab); free(db);
}

/*
 * Transpose of orc_rk4_step at the state (Phi, Pi) (the step's input): given lP, lQ (the
 * sensitivity to the step's output), overwrite them with the sensitivity to its input.
 */
void orc_rk4_step_vjp(int N, double dt, double sigma, const double *Phi, const double *Pi,
                      double *lP, double *lQ)
{
    size_t bytes = sizeof(double) * N;
    double *yP[4], *yQ[4], *kP = (double *)malloc(bytes), *kQ = (double *)malloc(bytes);
    double *A = (double *)malloc(bytes), *dl = (double *)malloc(bytes);
    double *kbP = (double *)malloc(bytes), *kbQ = (double *)malloc(bytes);
    double *ybP = (double *)malloc(bytes), *ybQ = (double *)malloc(bytes);
    double *inP = (double *)malloc(bytes), *inQ = (double *)malloc(bytes);
    const double cstage[4] = {0.0, 0.5, 0.5, 1.0};
    const double wstage[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    int st, i;
    /* recompute the stage inputs y_s exactly as the forward step does */
    for (st = 0; st < 4; ++st) {
        yP[st] = (double *)malloc(bytes);
        yQ[st] = (double *)malloc(bytes);
        if (st == 0) {
            memcpy(yP[0], Phi, bytes);
            memcpy(yQ[0], Pi, bytes);
        } else {
            for (i = 0; i < N; ++i) {
                yP[st][i] = Phi[i] + cstage[st] * dt * kP[i];
                yQ[st][i] = Pi[i] + cstage[st] * dt * kQ[i];
            }
        }
        orc_constraints(N, yP[st], yQ[st], A, dl, NULL, NULL);
        orc_rhs(N, sigma, yP[st], yQ[st], A, dl, kP, kQ);
    }
    /* reverse: kbar_s = w_s dt lambda + c_{s+1} dt ybar_{s+1};  ybar_s = R'(y_s)^T kbar_s */
    memcpy(inP, lP, bytes);
    memcpy(inQ, lQ, bytes);
    for (i = 0; i < N; ++i) { ybP[i] = 0.0; ybQ[i] = 0.0; }
    for (st = 3; st >= 0; --st) {
        for (i = 0; i < N; ++i) {
            kbP[i] = wstage[st] * dt * inP[i] + (st < 3 ? cstage[st + 1] * dt * ybP[i] : 0.0);
            kbQ[i] = wstage[st] * dt * inQ[i] + (st < 3 ? cstage[st + 1] * dt * ybQ[i] : 0.0);
            ybP[i] = 0.0;
            ybQ[i] = 0.0;
        }
        rhs_full_vjp(N, sigma, yP[st], yQ[st], kbP, kbQ, ybP, ybQ);
        for (i = 0; i < N; ++i) {
            lP[i] += ybP[i];
            lQ[i] += ybQ[i];
        }
    }
    for (st = 0; st < 4; ++st) { free(yP[st]); free(yQ[st]); }
    free(kP); free(kQ); free(A); free(dl); free(kbP); free(kbQ); free(ybP); free(ybQ);
    free(inP); free(inQ);
}

/*
 * Transpose of orc_spectrum (with A from orc_constraints of the same slice): given Ebar
 * (length J), accumulate the sensitivities to Phi and Pi.
 */
void orc_spectrum_vjp(int N, int J, const double *Phi, const double *Pi, const double *Ebar,
                      double *Phibar, double *Pibar)
{
    const double h = grid_h(N);
    double *A = (double *)malloc(sizeof(double) * N), *dl = (double *)malloc(sizeof(double) * N);
    double *Ab = (double *)calloc(N, sizeof(double)), *db = (double *)calloc(N, sizeof(double));
    double *e = (double *)malloc(sizeof(double) * (size_t)N * J);
    double *de = (double *)malloc(sizeof(double) * (size_t)N * J);
    int j, i;
    orc_constraints(N, Phi, Pi, A, dl, NULL, NULL);
    orc_eigen(N, J, e, de);
    for (j = 0; j < J; ++j) {
        double pj = 0.0, fj = 0.0, om = 3.0 + 2.0 * j, pb, fb;
        for (i = 1; i < N - 1; ++i) {
            double x = i * h, t2 = tan(x) * tan(x), sa = sqrt(A[i]);
            pj += h * t2 * sa * Pi[i] * e[(size_t)j * N + i];
            fj += h * t2 * sa * Phi[i] * de[(size_t)j * N + i];
        }
        pb = 2.0 * pj * Ebar[j];
        fb = 2.0 * fj * Ebar[j] / (om * om);
        for (i = 1; i < N - 1; ++i) {
            double x = i * h, t2 = tan(x) * tan(x), sa = sqrt(A[i]);
            Pibar[i] += pb * h * t2 * sa * e[(size_t)j * N + i];
            Phibar[i] += fb * h * t2 * sa * de[(size_t)j * N + i];
            Ab[i] += (pb * h * t2 * Pi[i] * e[(size_t)j * N + i]
                      + fb * h * t2 * Phi[i] * de[(size_t)j * N + i]) / (2.0 * sa);
        }
    }
    orc_constraints_vjp(N, Phi, Pi, Ab, db, Phibar, Pibar);
    free(A); free(dl); free(Ab); free(db); free(e); free(de);
}

/*
 * The mode-energy drift functional J = sum_{j<Jm} (E_j(T) - E_j(0))^2 of an evolution from
 * Pi(x,0) = sum_{k<K} a_k e_k, Phi(x,0) = 0 over nsteps RK4 steps of size dt (no collapse
 * stop), and its gradient dJ/da by the discrete adjoint: states stored every step, one
 * backward sweep.  out[0] = J; dJda has length K.
 */
void orc_grad(int N, int K, const double *a, long nsteps, double dt, double sigma, int Jm,
              double *out, double *dJda)
{
    size_t bytes = sizeof(double) * N;
    double *P = (double *)malloc(bytes * (nsteps + 1)), *Q = (double *)malloc(bytes * (nsteps + 1));
    double *A = (double *)malloc(bytes), *dl = (double *)malloc(bytes);
    double *E0 = (double *)malloc(sizeof(double) * Jm), *ET = (double *)malloc(sizeof(double) * Jm);
    double *Eb = (double *)malloc(sizeof(double) * Jm);
    double *lP = (double *)calloc(N, sizeof(double)), *lQ = (double *)calloc(N, sizeof(double));
    double *e = (double *)malloc(sizeof(double) * (size_t)N * K);
    double *de = (double *)malloc(sizeof(double) * (size_t)N * K);
    double Jv = 0.0;
    long n;
    int j, i;
    orc_synthesize(N, K, a, P, Q);
    for (n = 0; n < nsteps; ++n) {
        memcpy(P + (n + 1) * N, P + n * N, bytes);
        memcpy(Q + (n + 1) * N, Q + n * N, bytes);
        orc_rk4_step(N, dt, sigma, P + (n + 1) * N, Q + (n + 1) * N);
    }
    orc_constraints(N, P, Q, A, dl, NULL, NULL);
    orc_spectrum(N, Jm, P, Q, A, E0, NULL, NULL);
    orc_constraints(N, P + nsteps * N, Q + nsteps * N, A, dl, NULL, NULL);
    orc_spectrum(N, Jm, P + nsteps * N, Q + nsteps * N, A, ET, NULL, NULL);
    for (j = 0; j < Jm; ++j) Jv += (ET[j] - E0[j]) * (ET[j] - E0[j]);
    out[0] = Jv;
    /* J through E(T) */
    for (j = 0; j < Jm; ++j) Eb[j] = 2.0 * (ET[j] - E0[j]);
    orc_spectrum_vjp(N, Jm, P + nsteps * N, Q + nsteps * N, Eb, lP, lQ);
    for (n = nsteps - 1; n >= 0; --n) orc_rk4_step_vjp(N, dt, sigma, P + n * N, Q + n * N, lP, lQ);
    /* J through E(0) */
    for (j = 0; j < Jm; ++j) Eb[j] = -2.0 * (ET[j] - E0[j]);
    orc_spectrum_vjp(N, Jm, P, Q, Eb, lP, lQ);
    /* Pi(x,0) = sum_k a_k e_k with Pi_{N-1} = 0 imposed; Phi(x,0) = 0 does not depend on a */
    orc_eigen(N, K, e, de);
    for (j = 0; j < K; ++j) {
        double s = 0.0;
        for (i = 0; i < N - 1; ++i) s += lQ[i] * e[(size_t)j * N + i];
        dJda[j] = s;
    }
    free(P); free(Q); free(A); free(dl); free(E0); free(ET); free(Eb); free(lP); free(lQ);
    free(e); free(de);
}
