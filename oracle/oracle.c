/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY. Not part of the product path.
 *
 * A plain, slow, one-system-at-a-time FP64 CPU restatement of the method of
 * F. Hegedus, "Modular, general purpose ODE integration package to solve large
 * number of independent ODE systems on GPUs" (arXiv:1810.03931): per-system
 * integration with the classic fourth-order Runge-Kutta scheme (fixed step) or
 * the adaptive Runge-Kutta-Cash-Karp 4(5) scheme (Sec. 3), the event
 * handling state machine (Sec. 4, Sec. 6.6), accessories (Sec. 5, Sec. 6.7),
 * initialization / finalization hooks (Sec. 6.8) and the three test models of
 * Sec. 2 (Duffing Eqs. (1)-(2), Keller-Miksis Eqs. (12)-(28), pressure relief
 * valve Eqs. (29)-(34)), the Duffing equation extended by its linearisation
 * in polar coordinates for the largest Lyapunov exponent (Eqs. (3)-(7)), plus
 * a bouncing ball used only for closed-form pins.
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's library. It shares no code with the CUDA library and neither
 * includes nor links the other. Build with -ffp-contract=off so that every
 * a*b+c below rounds twice, exactly as written.
 *
 * Array layout of every per-system quantity is structure-of-arrays,
 * value[component * N + system], as the problem pool of Sec. 6.1 prescribes.
 *
 * Readings of points where the paper is silent or ambiguous (they are listed
 * with reasons in the design notes of the repository):
 *  - Cash-Karp coefficients are those published by Cash & Karp (ACM TOMS 16,
 *    1990, 201-222); the fifth-order solution is propagated (local
 *    extrapolation); the difference to the embedded fourth-order solution is
 *    the local error estimate (Sec. 3).
 *  - Error ratio: max_i |e_i| / (atol_i + rtol_i * max(|y_n,i|, |y_n+1,i|));
 *    accept when <= 1; new step h * clamp(0.9 * err^(-1/5), shrink, grow),
 *    clamped to [hmin, hmax]; err == 0 gives the grow limit (Sec. 6.5).
 *  - At hmin a step is accepted whatever its error; a non-finite error rejects
 *    the step and shrinks h, and a non-finite error at hmin stops the system
 *    (Sec. 6.5).
 *  - The last step of a slice is clipped so that the slice ends exactly at t1.
 *  - Events: a crossing in the allowed direction (MATLAB rule, Sec. 6.6) from
 *    outside the zone |F| <= tol is detected; a point inside the zone ends the
 *    search at once, otherwise the crossing is located by bisection in the step
 *    size, re-stepping from the last accepted point, until |F| <= tol (Sec. 4;
 *    the paper's secant search is replaced by bisection).  Only the event with
 *    the largest index is located; the others fire at the located point if
 *    they are still crossed there (Sec. 4).
 *  - Event counters are 1-based and restart at every slice (Sec. 6.7, 7.2).
 *  - Hook order after an accepted step: ordinary accessories, then for each
 *    detected event in ascending order: counter, event accessories, event
 *    action; then the zone bookkeeping and the stop checks.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_MAXN 4
#define ORC_MAXP 16
#define ORC_MAXA 8
#define ORC_MAXE 2

enum { ORC_DUFFING = 0, ORC_KELLER_MIKSIS = 1, ORC_VALVE = 2, ORC_BOUNCE = 3,
       ORC_DUFFING_LYAPUNOV = 4 };
enum { ORC_RK4 = 0, ORC_RKCK45 = 1 };
enum { ORC_TD_KEEP = 0, ORC_TD_T0_TO_T = 1, ORC_TD_SHIFT = 2 };
enum {
    ORC_ST_NONE = 0,
    ORC_ST_TEND = 1,
    ORC_ST_EVENT_STOP = 2,
    ORC_ST_EQUILIBRIUM = 3,
    ORC_ST_HMIN_NAN = 4,
    ORC_ST_STEP_BUDGET = 5
};

/* Solver-wide settings: the ODE properties of Sec. 6.5, the event properties
 * of Sec. 6.6 and the solver configuration of Sec. 6.4. */
typedef struct orc_config {
    int model;
    int scheme;
    int events_on;
    int td_mode;
    double h0;
    double rtol[ORC_MAXN];
    double atol[ORC_MAXN];
    double hmax, hmin, grow, shrink;
    int evt_dir[ORC_MAXE];
    double evt_tol[ORC_MAXE];
    int evt_stop[ORC_MAXE];
    int max_eq;
    long long max_steps;
    double mc[8];
} orc_config;

/* Optional per-step trace of one system (tests only). */
typedef struct orc_trace {
    int cap;
    int n_points;      /* accepted points written to t[] / y[] */
    double *t;         /* [cap] */
    double *y;         /* [cap * ORC_MAXN] */
    int ev_cap;
    int n_events;
    int *ev_index;     /* [ev_cap] */
    double *ev_t;      /* [ev_cap] */
    double *ev_y;      /* [ev_cap * ORC_MAXN], state before the action */
    double *ev_y_after; /* [ev_cap * ORC_MAXN], state after it (may be NULL) */
    /* trial steps of the adaptive scheme (all may be NULL / 0) */
    int trial_cap;
    int n_trials;
    double *trial_t;     /* [trial_cap] start time of the trial */
    double *trial_h;     /* [trial_cap] its step size */
    double *trial_y;     /* [trial_cap * ORC_MAXN] state at the start */
    double *trial_ynew;  /* [trial_cap * ORC_MAXN] fifth-order result */
    double *trial_e;     /* [trial_cap * ORC_MAXN] embedded error estimate */
    int *trial_ok;       /* [trial_cap] 1 accepted, 0 rejected, -1 non-finite */
    double *trial_hnext; /* [trial_cap] step size the controller chose next */
} orc_trace;

/* Record one trial step of the adaptive scheme in the trace (tests only). */
static void record_trial(orc_trace *tr, int n, double t, double hs, const double *y,
                         const double *ynew, const double *e, int ok, double hnext)
{
    if (!tr || !tr->trial_t || tr->n_trials >= tr->trial_cap) return;
    int k = tr->n_trials++;
    tr->trial_t[k] = t;
    tr->trial_h[k] = hs;
    for (int m = 0; m < n; m++) {
        tr->trial_y[k * ORC_MAXN + m] = y[m];
        tr->trial_ynew[k * ORC_MAXN + m] = ynew[m];
        tr->trial_e[k * ORC_MAXN + m] = e[m];
    }
    tr->trial_ok[k] = ok;
    tr->trial_hnext[k] = hnext;
}

/* ------------------------------------------------------------------------ */
/* Model dimensions (Sec. 2 and the hooks of Sec. 6.5-6.8).                  */
/* ------------------------------------------------------------------------ */
int orc_dims(int model, int *n, int *P, int *A, int *E)
{
    switch (model) {
    case ORC_DUFFING:       *n = 2; *P = 2;  *A = 7; *E = 1; return 0;
    case ORC_KELLER_MIKSIS: *n = 2; *P = 13; *A = 4; *E = 1; return 0;
    case ORC_VALVE:         *n = 3; *P = 5;  *A = 5; *E = 2; return 0;
    case ORC_BOUNCE:        *n = 2; *P = 2;  *A = 6; *E = 1; return 0;
    case ORC_DUFFING_LYAPUNOV: *n = 4; *P = 2; *A = 5; *E = 1; return 0;
    default: return -1;
    }
}

/* ------------------------------------------------------------------------ */
/* Right-hand sides f(y, t; p), Eq. (38).                                    */
/* ------------------------------------------------------------------------ */

/* Duffing, Eqs. (1)-(2): y1' = y2, y2' = delta*y1 - c3*y1^3 - k*y2 + B*cos(w t).
 * Per-system parameters p = (k, B); solver constants mc = (delta, c3, w). */
static void rhs_duffing(const orc_config *c, double t, const double *y,
                        const double *p, double *f)
{
    double delta = c->mc[0], c3 = c->mc[1], w = c->mc[2];
    double k = p[0], B = p[1];
    f[0] = y[1];
    f[1] = delta * y[0] - c3 * y[0] * y[0] * y[0] - k * y[1] + B * cos(w * t);
}

/* Duffing with its linearisation attached in polar coordinates, Eqs. (3)-(6):
 * y3 is the radius and y4 the angle of a tangent vector of (y1, y2),
 *   y3' = y3 ((1 + g1) sin(y4) cos(y4) + g2 sin(y4)^2),
 *   y4' = -sin(y4)^2 + (g1 cos(y4) + g2 sin(y4)) cos(y4),
 * with g1 = dF2/dy1 = delta - 3 c3 y1^2 and g2 = dF2/dy2 = -k, F2 the
 * right-hand side of y2.  Same p and mc as the Duffing model. */
static void rhs_duffing_lyapunov(const orc_config *c, double t, const double *y,
                                 const double *p, double *f)
{
    double delta = c->mc[0], c3 = c->mc[1];
    double k = p[0];
    rhs_duffing(c, t, y, p, f);
    double g1 = delta - 3.0 * c3 * y[0] * y[0];
    double g2 = -k;
    double s = sin(y[3]), co = cos(y[3]);
    f[2] = y[2] * ((1.0 + g1) * s * co + g2 * s * s);
    f[3] = -s * s + (g1 * co + g2 * s) * co;
}

/* Keller-Miksis in the dimensionless form of Eqs. (12)-(15); p = C0..C12 of
 * Eqs. (16)-(28); t is the dimensionless time tau. */
static void rhs_keller_miksis(double tau, const double *y, const double *C,
                              double *f)
{
    const double two_pi = 2.0 * M_PI;
    double y1 = y[0], y2 = y[1];
    double rx = 1.0 / y1;
    double s1 = sin(two_pi * tau);
    double c1 = cos(two_pi * tau);
    double s2 = sin(two_pi * C[11] * tau + C[12]);
    double c2 = cos(two_pi * C[11] * tau + C[12]);
    double num = (C[0] + C[1] * y2) * pow(rx, C[10])
               - C[2] * (1.0 + C[9] * y2)
               - C[3] * rx
               - C[4] * y2 * rx
               - (1.0 - C[9] * y2 / 3.0) * 1.5 * y2 * y2
               - (C[5] * s1 + C[6] * s2) * (1.0 + C[9] * y2)
               - y1 * (C[7] * c1 + C[8] * c2);
    double den = y1 - C[9] * y1 * y2 + C[4] * C[9];
    f[0] = y2;
    f[1] = num / den;
}

/* Pressure relief valve, Eqs. (29)-(31); p = (kappa, delta, beta, q, r). */
static void rhs_valve(const double *y, const double *p, double *f)
{
    double kappa = p[0], delta = p[1], beta = p[2], q = p[3];
    f[0] = y[1];
    f[1] = -kappa * y[1] - (y[0] + delta) + y[2];
    f[2] = beta * (q - y[0] * sqrt(y[2]));
}

/* Bouncing ball (pins only): y1' = y2, y2' = -g; p = (g, r). */
static void rhs_bounce(const double *y, const double *p, double *f)
{
    f[0] = y[1];
    f[1] = -p[0];
}

static void rhs(const orc_config *c, double t, const double *y,
                const double *p, double *f)
{
    switch (c->model) {
    case ORC_DUFFING:       rhs_duffing(c, t, y, p, f); break;
    case ORC_KELLER_MIKSIS: rhs_keller_miksis(t, y, p, f); break;
    case ORC_VALVE:         rhs_valve(y, p, f); break;
    case ORC_DUFFING_LYAPUNOV: rhs_duffing_lyapunov(c, t, y, p, f); break;
    default:                rhs_bounce(y, p, f); break;
    }
}

/* ------------------------------------------------------------------------ */
/* Event functions F_Ej(y, t) = 0, Eqs. (35)-(37), and actions (Sec. 6.6).   */
/* ------------------------------------------------------------------------ */
static void event_functions(const orc_config *c, double t, const double *y,
                            const double *p, double *F)
{
    (void)t; (void)p;
    switch (c->model) {
    case ORC_DUFFING:       F[0] = y[1]; break;             /* extrema of y1 */
    case ORC_KELLER_MIKSIS: F[0] = y[1]; break;
    case ORC_VALVE:         F[0] = y[1]; F[1] = y[0]; break; /* max, impact */
    case ORC_DUFFING_LYAPUNOV: F[0] = y[1]; break;
    default:                F[0] = y[0]; break;             /* ball on floor */
    }
}

/* Event action: the impact law of Eqs. (32)-(34), y2+ = -r * y2-. */
static void event_action(const orc_config *c, int j, double *y, const double *p)
{
    if (c->model == ORC_VALVE && j == 1)
        y[1] = -p[4] * y[1];
    if (c->model == ORC_BOUNCE && j == 0)
        y[1] = -p[1] * y[1];
}

/* ------------------------------------------------------------------------ */
/* Accessories (Sec. 5, Sec. 6.7) and initialization (Sec. 6.8).             */
/*  all models: a0 = max y1, a1 = its time, a2 = min y1, a3 = its time       */
/*  Duffing:    a4, a5 = y1 and t at the first detection of event 0,         */
/*              a6 = number of detections of event 0                          */
/*  valve:      a4 = number of impacts (event 1)                             */
/*  ball:       a4 = time of the last impact, a5 = velocity before it        */
/*  Lyapunov:   a4 = ln y3 at the end of the slice (Finalization, below)      */
/* ------------------------------------------------------------------------ */
static void acc_initialization(const orc_config *c, double t, const double *y,
                               double *a)
{
    a[0] = y[0]; a[1] = t; a[2] = y[0]; a[3] = t;
    switch (c->model) {
    case ORC_DUFFING: a[4] = y[0]; a[5] = t; a[6] = 0.0; break;
    case ORC_VALVE:   a[4] = 0.0; break;
    case ORC_BOUNCE:  a[4] = t; a[5] = y[1]; break;
    case ORC_DUFFING_LYAPUNOV: a[4] = 0.0; break;
    default: break;
    }
}

static void acc_ordinary(double t, const double *y, double *a)
{
    if (y[0] > a[0]) { a[0] = y[0]; a[1] = t; }
    if (y[0] < a[2]) { a[2] = y[0]; a[3] = t; }
}

static void acc_event(const orc_config *c, int j, int counter, double t,
                      const double *y, double *a)
{
    if (c->model == ORC_DUFFING && j == 0) {
        a[6] = (double)counter;
        if (counter == 1) { a[4] = y[0]; a[5] = t; }
    } else if (c->model == ORC_VALVE && j == 1) {
        a[4] = (double)counter;
    } else if (c->model == ORC_BOUNCE && j == 0) {
        a[4] = t; a[5] = y[1];
    }
}

/* ------------------------------------------------------------------------ */
/* Butcher tableaux (Sec. 3).                                                */
/* ------------------------------------------------------------------------ */

/* Cash & Karp (1990), embedded 4(5) pair. */
static const double CK_C[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double CK_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0},
};
/* fifth-order weights (propagated) and embedded fourth-order weights */
static const double CK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static const double CK_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                                277.0 / 14336.0, 1.0 / 4.0};

/* Classic fourth-order Runge-Kutta. */
static const double RK4_C[4] = {0.0, 0.5, 0.5, 1.0};
static const double RK4_A[4][3] = {{0, 0, 0}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 1.0}};
static const double RK4_B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

/* Export the Cash-Karp tableau for the order-condition test:
 * c[6], a[6*6] row-major (zero above the diagonal), b5[6], b4[6]. */
void orc_ck_tableau(double *c, double *a, double *b5, double *b4)
{
    for (int i = 0; i < 6; i++) {
        c[i] = CK_C[i];
        b5[i] = CK_B5[i];
        b4[i] = CK_B4[i];
        for (int j = 0; j < 6; j++)
            a[i * 6 + j] = (j < 5) ? CK_A[i][j] : 0.0;
    }
}

void orc_rk4_tableau(double *c, double *a, double *b)
{
    for (int i = 0; i < 4; i++) {
        c[i] = RK4_C[i];
        b[i] = RK4_B[i];
        for (int j = 0; j < 4; j++)
            a[i * 4 + j] = (j < 3) ? RK4_A[i][j] : 0.0;
    }
}

/* One explicit Runge-Kutta step of size h from (t, y):
 *   k_i = f(t + c_i h, y + h sum_j a_ij k_j),  y_new = y + h sum_i b_i k_i,
 * and for Cash-Karp the error estimate e = h sum_i (b5_i - b4_i) k_i. */
static void rk_step(const orc_config *c, int n, double t, const double *y,
                    const double *p, double h, double *ynew, double *err)
{
    double k[6][ORC_MAXN];
    double ys[ORC_MAXN];
    int stages = (c->scheme == ORC_RK4) ? 4 : 6;
    for (int i = 0; i < stages; i++) {
        for (int m = 0; m < n; m++) {
            double s = 0.0;
            for (int j = 0; j < i; j++) {
                double aij = (c->scheme == ORC_RK4) ? RK4_A[i][j] : CK_A[i][j];
                s += aij * k[j][m];
            }
            ys[m] = y[m] + h * s;
        }
        double ci = (c->scheme == ORC_RK4) ? RK4_C[i] : CK_C[i];
        rhs(c, t + ci * h, ys, p, k[i]);
    }
    for (int m = 0; m < n; m++) {
        double s = 0.0, e = 0.0;
        for (int i = 0; i < stages; i++) {
            if (c->scheme == ORC_RK4) {
                s += RK4_B[i] * k[i][m];
            } else {
                s += CK_B5[i] * k[i][m];
                e += (CK_B5[i] - CK_B4[i]) * k[i][m];
            }
        }
        ynew[m] = y[m] + h * s;
        if (err) err[m] = h * e;
    }
}

static int all_finite(int n, const double *v)
{
    for (int m = 0; m < n; m++)
        if (!isfinite(v[m])) return 0;
    return 1;
}

static double clampd(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

/* Does event j cross in its allowed direction between F_old (outside the
 * zone) and F_new?  Landing inside the zone counts as a crossing. */
static int crossed(const orc_config *c, int j, double F_old, double F_new)
{
    double tol = c->evt_tol[j];
    int down = (F_old > 0.0) && (F_new <= tol);
    int up = (F_old < 0.0) && (F_new >= -tol);
    int dir = c->evt_dir[j];
    if (dir < 0) return down;
    if (dir > 0) return up;
    return down || up;
}

/* ------------------------------------------------------------------------ */
/* One integration phase (one call of Solve, Sec. 6.4) of one system.        */
/* Returns the stop reason.                                                  */
/* ------------------------------------------------------------------------ */
static int integrate_slice(const orc_config *c, int n, int A, int E,
                           double *td, double *y, const double *p, double *a,
                           int *ecnt, long long *nacc, long long *nrej,
                           double *t_end, orc_trace *tr)
{
    double t0 = td[0], t1 = td[1];
    double t = t0;
    (void)A;

    /* Initialization hook (Sec. 6.8). */
    acc_initialization(c, t, y, a);
    if (tr && tr->n_points < tr->cap) {
        tr->t[tr->n_points] = t;
        for (int m = 0; m < n; m++) tr->y[tr->n_points * ORC_MAXN + m] = y[m];
        tr->n_points++;
    }

    /* Event state at t0: a point already inside a zone is in the leaving
     * state and is not detected (Sec. 4, Sec. 7.2). */
    int nE = c->events_on ? E : 0;
    double F[ORC_MAXE];
    int leaving[ORC_MAXE], inzone[ORC_MAXE];
    if (nE > 0) event_functions(c, t, y, p, F);
    for (int j = 0; j < nE; j++) {
        ecnt[j] = 0;
        leaving[j] = fabs(F[j]) <= c->evt_tol[j];
        inzone[j] = 0;
    }

    /* Step size: RK4 divides the slice into equal steps no longer than h0;
     * RKCK45 starts from the prescribed initial step (Sec. 6.4). */
    double h;
    if (c->scheme == ORC_RK4) {
        double nsteps = ceil((t1 - t0) / c->h0 - 1e-9);
        if (nsteps < 1.0) nsteps = 1.0;
        h = (t1 - t0) / nsteps;
    } else {
        h = clampd(c->h0, c->hmin, c->hmax);
    }

    int status = ORC_ST_NONE;
    long long steps = 0;
    if (!(t < t1)) status = ORC_ST_TEND;

    while (status == ORC_ST_NONE) {
        if (steps >= c->max_steps) { status = ORC_ST_STEP_BUDGET; break; }

        /* Clip the last step to the end of the time domain; a remainder
         * within 1e-9 h of a full step is taken as the last step, so that
         * rounding in t never leaves a sliver step. */
        double hs = h;
        int last = 0;
        if (t1 - t <= hs * (1.0 + 1e-9)) {
            hs = t1 - t;
            last = 1;
        }

        double ynew[ORC_MAXN], e[ORC_MAXN];
        rk_step(c, n, t, y, p, hs, ynew, e);
        steps++;

        double hnext = h;
        if (c->scheme == ORC_RKCK45) {
            /* Error ratio and step-size control (Sec. 3, Sec. 6.5). */
            double err = 0.0;
            for (int m = 0; m < n; m++) {
                double sc = c->atol[m] + c->rtol[m] * fmax(fabs(y[m]), fabs(ynew[m]));
                double r = fabs(e[m]) / sc;
                if (r > err || isnan(r)) err = r;
            }
            int at_min = hs <= c->hmin;
            if (!isfinite(err) || !all_finite(n, ynew)) {
                (*nrej)++;
                if (at_min) {
                    record_trial(tr, n, t, hs, y, ynew, e, -1, hs);
                    status = ORC_ST_HMIN_NAN;
                    break;
                }
                h = fmax(c->shrink * hs, c->hmin);
                record_trial(tr, n, t, hs, y, ynew, e, -1, h);
                continue;
            }
            double fac = (err == 0.0) ? c->grow : 0.9 * pow(err, -0.2);
            fac = clampd(fac, c->shrink, c->grow);
            if (err > 1.0 && !at_min) {
                (*nrej)++;
                h = clampd(hs * fac, c->hmin, c->hmax);
                record_trial(tr, n, t, hs, y, ynew, e, 0, h);
                continue;
            }
            hnext = clampd(hs * fac, c->hmin, c->hmax);
            record_trial(tr, n, t, hs, y, ynew, e, 1, hnext);
        } else if (!all_finite(n, ynew)) {
            /* the fixed RK4 step is also the minimum step */
            (*nrej)++;
            status = ORC_ST_HMIN_NAN;
            break;
        }

        double tnew = last ? t1 : t + hs;
        int located = 0;

        /* Event detection and location (Sec. 4, Sec. 6.6). */
        int det[ORC_MAXE] = {0};
        if (nE > 0) {
            double Fn[ORC_MAXE];
            event_functions(c, tnew, ynew, p, Fn);
            int jstar = -1;
            for (int j = 0; j < nE; j++) {
                if (!leaving[j] && crossed(c, j, F[j], Fn[j])) {
                    det[j] = 1;
                    jstar = j;
                }
            }
            if (jstar >= 0 && fabs(Fn[jstar]) > c->evt_tol[jstar]) {
                /* Configuration a: the step jumped over the zone.  Bisect the
                 * step size, re-stepping from the accepted point (t, y). */
                double lo = 0.0, hi = hs;
                double yhi[ORC_MAXN];
                for (int m = 0; m < n; m++) yhi[m] = ynew[m];
                int pre_sign = F[jstar] > 0.0 ? 1 : -1;
                for (int it = 0; it < 200; it++) {
                    double mid = 0.5 * (lo + hi);
                    if (mid <= lo || mid >= hi) break;
                    double ym[ORC_MAXN], Fm[ORC_MAXE];
                    rk_step(c, n, t, y, p, mid, ym, NULL);
                    event_functions(c, t + mid, ym, p, Fm);
                    if (fabs(Fm[jstar]) <= c->evt_tol[jstar]) {
                        hi = mid;
                        for (int m = 0; m < n; m++) yhi[m] = ym[m];
                        break;
                    }
                    if ((Fm[jstar] > 0.0 ? 1 : -1) == pre_sign) {
                        lo = mid;
                    } else {
                        hi = mid;
                        for (int m = 0; m < n; m++) yhi[m] = ym[m];
                    }
                }
                tnew = t + hi;
                for (int m = 0; m < n; m++) ynew[m] = yhi[m];
                located = 1;
                /* The other events fire at the located point only if they are
                 * crossed there as well. */
                event_functions(c, tnew, ynew, p, Fn);
                for (int j = 0; j < nE; j++)
                    if (j != jstar)
                        det[j] = det[j] && crossed(c, j, F[j], Fn[j]);
            }
        }

        /* Accept the step. */
        t = tnew;
        for (int m = 0; m < n; m++) y[m] = ynew[m];
        (*nacc)++;
        if (c->scheme == ORC_RKCK45) h = hnext;
        if (tr && tr->n_points < tr->cap) {
            tr->t[tr->n_points] = t;
            for (int m = 0; m < n; m++) tr->y[tr->n_points * ORC_MAXN + m] = y[m];
            tr->n_points++;
        }

        /* Ordinary accessories at every accepted step (Sec. 6.7). */
        acc_ordinary(t, y, a);

        if (nE > 0) {
            /* Detected events in ascending order: counter, event
             * accessories, action (Sec. 6.6, 6.7). */
            for (int j = 0; j < nE; j++) {
                if (!det[j]) continue;
                ecnt[j]++;
                if (tr && tr->n_events < tr->ev_cap) {
                    tr->ev_index[tr->n_events] = j;
                    tr->ev_t[tr->n_events] = t;
                    for (int m = 0; m < n; m++) tr->ev_y[tr->n_events * ORC_MAXN + m] = y[m];
                    tr->n_events++;
                }
                acc_event(c, j, ecnt[j], t, y, a);
                event_action(c, j, y, p);
                if (tr && tr->ev_y_after && tr->n_events > 0 && tr->n_events <= tr->ev_cap)
                    for (int m = 0; m < n; m++)
                        tr->ev_y_after[(tr->n_events - 1) * ORC_MAXN + m] = y[m];
            }
            /* Zone bookkeeping at the (post-action) accepted point. */
            event_functions(c, t, y, p, F);
            for (int j = 0; j < nE; j++) {
                int in_zone = fabs(F[j]) <= c->evt_tol[j];
                if (det[j]) {
                    leaving[j] = 1;
                    inzone[j] = 0;
                } else if (leaving[j]) {
                    if (!in_zone) {
                        leaving[j] = 0;
                        inzone[j] = 0;
                    } else {
                        inzone[j]++;
                        if (c->max_eq > 0 && inzone[j] >= c->max_eq)
                            status = ORC_ST_EQUILIBRIUM;
                    }
                } else if (in_zone) {
                    leaving[j] = 1;
                    inzone[j] = 0;
                }
            }
            for (int j = 0; j < nE; j++)
                if (det[j] && c->evt_stop[j] > 0 && ecnt[j] >= c->evt_stop[j])
                    status = ORC_ST_EVENT_STOP;
        }

        if (status == ORC_ST_NONE && last && !located)
            status = ORC_ST_TEND;
    }

    *t_end = t;
    /* Finalization hook (Sec. 6.8): time-domain update chosen per solver. */
    if (c->td_mode == ORC_TD_T0_TO_T) {
        td[0] = t;
    } else if (c->td_mode == ORC_TD_SHIFT) {
        double span = t1 - t0;
        td[0] = t;
        td[1] = t + span;
    }
    /* Lyapunov model: the stretch of the tangent vector over the slice is
     * kept as ln y3 and the radius restarts from one (Sec. 2.1, Eq. (7):
     * y3 is reset at every Poincare point t_n; the exponent is the mean of
     * ln y3(t_n) per unit time -- the printed Eq. (7) averages y3 itself).
     * The angle is brought back to [-pi, pi]: Eqs. (3)-(4) see it only
     * through sin and cos, and an angle that winds without bound would
     * loosen its relative tolerance (the paper is silent on this). */
    if (c->model == ORC_DUFFING_LYAPUNOV) {
        a[4] = log(y[2]);
        y[2] = 1.0;
        y[3] = remainder(y[3], 2.0 * M_PI);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Driver: n_slices consecutive calls of Solve for every system (the loop of */
/* Sec. 7.1.1), the last (n_slices - n_skip) of them recorded.               */
/* Record layout: records[((s - n_skip) * R + comp) * N + i], R = A + n + 1, */
/* comp = accessories, then end state, then end time.                        */
/* ------------------------------------------------------------------------ */
typedef struct orc_job {
    const orc_config *c;
    int N, n, A, E, P;
    double *td, *y, *acc, *records;
    const double *p;
    int *status, *ecnt;
    long long *nacc, *nrej;
    int n_slices, n_skip;
    int i_begin, i_end;
} orc_job;

static void run_system(const orc_job *jb, int i)
{
    const int N = jb->N, n = jb->n, A = jb->A, E = jb->E, P = jb->P;
    double td[2], y[ORC_MAXN], p[ORC_MAXP], a[ORC_MAXA];
    int ecnt[ORC_MAXE] = {0};
    long long nacc = 0, nrej = 0;
    td[0] = jb->td[i];
    td[1] = jb->td[N + i];
    for (int m = 0; m < n; m++) y[m] = jb->y[m * N + i];
    for (int m = 0; m < P; m++) p[m] = jb->p[m * N + i];
    for (int m = 0; m < A; m++) a[m] = jb->acc[m * N + i];
    int st = ORC_ST_NONE;
    const int R = A + n + 1;
    for (int s = 0; s < jb->n_slices; s++) {
        double t_end;
        st = integrate_slice(jb->c, n, A, E, td, y, p, a, ecnt, &nacc, &nrej, &t_end, NULL);
        if (jb->records && s >= jb->n_skip) {
            long long r = s - jb->n_skip;
            double *rec = jb->records;
            for (int m = 0; m < A; m++) rec[(r * R + m) * N + i] = a[m];
            for (int m = 0; m < n; m++) rec[(r * R + A + m) * N + i] = y[m];
            rec[(r * R + A + n) * N + i] = t_end;
        }
    }
    jb->td[i] = td[0];
    jb->td[N + i] = td[1];
    for (int m = 0; m < n; m++) jb->y[m * N + i] = y[m];
    for (int m = 0; m < A; m++) jb->acc[m * N + i] = a[m];
    if (jb->status) jb->status[i] = st;
    if (jb->ecnt)
        for (int j = 0; j < E; j++) jb->ecnt[j * N + i] = jb->c->events_on ? ecnt[j] : 0;
    if (jb->nacc) jb->nacc[i] += nacc;
    if (jb->nrej) jb->nrej[i] += nrej;
}

static void *run_range(void *arg)
{
    const orc_job *jb = (const orc_job *)arg;
    for (int i = jb->i_begin; i < jb->i_end; i++) run_system(jb, i);
    return NULL;
}

/* Integrate N systems over n_slices consecutive slices.  nthreads > 1 splits
 * the systems into contiguous ranges, one POSIX thread each (the arithmetic
 * of every system is unchanged). */
int orc_run(const orc_config *c, int N, double *td, double *y, const double *p,
            double *acc, int *status, int *ecnt, long long *nacc,
            long long *nrej, int n_slices, int n_skip, double *records,
            int nthreads)
{
    int n, P, A, E;
    if (orc_dims(c->model, &n, &P, &A, &E) != 0) return -1;
    if (N < 0 || n_slices < 0 || n_skip < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > N) nthreads = N > 0 ? N : 1;
    orc_job base = {c, N, n, A, E, P, td, y, acc, records, p, status, ecnt,
                    nacc, nrej, n_slices, n_skip, 0, N};
    if (nthreads == 1) {
        run_range(&base);
        return 0;
    }
    pthread_t th[256];
    orc_job jobs[256];
    for (int k = 0; k < nthreads; k++) {
        jobs[k] = base;
        jobs[k].i_begin = (int)((long long)N * k / nthreads);
        jobs[k].i_end = (int)((long long)N * (k + 1) / nthreads);
        if (pthread_create(&th[k], NULL, run_range, &jobs[k]) != 0) {
            run_range(&jobs[k]);
            th[k] = 0;
        }
    }
    for (int k = 0; k < nthreads; k++)
        if (th[k]) pthread_join(th[k], NULL);
    return 0;
}

/* One slice of one system with a trace of accepted points and events
 * (tests only).  State arrays are plain vectors (N = 1). */
int orc_trace_slice(const orc_config *c, double *td, double *y, const double *p,
                    double *acc, int *ecnt, long long *nacc, long long *nrej,
                    orc_trace *tr)
{
    int n, P, A, E;
    if (orc_dims(c->model, &n, &P, &A, &E) != 0) return -1;
    double t_end;
    return integrate_slice(c, n, A, E, td, y, p, acc, ecnt, nacc, nrej, &t_end, tr);
}

/* One explicit step (tests only): exposes the stage arithmetic for the
 * observed-order pins.  err may be NULL. */
int orc_single_step(const orc_config *c, double t, const double *y,
                    const double *p, double h, double *ynew, double *err)
{
    int n, P, A, E;
    if (orc_dims(c->model, &n, &P, &A, &E) != 0) return -1;
    rk_step(c, n, t, y, p, h, ynew, err);
    return 0;
}

int orc_rhs(const orc_config *c, double t, const double *y, const double *p,
            double *f)
{
    rhs(c, t, y, p, f);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Keller-Miksis coefficients C0..C12, Eqs. (16)-(28), from the physical     */
/* parameters of Sec. 2.2 (SI units; omega in rad/s).  Eq. (24) prints C8    */
/* with omega_1; the time derivative of P_A2 sin(omega_2 t) in Eq. (8) gives */
/* omega_2, which is what is used (an independent integration of the         */
/* dimensional Eqs. (8)-(11) with two frequencies agrees only with omega_2). */
/* ------------------------------------------------------------------------ */
void orc_km_coefficients(double PA1, double PA2, double omega1, double omega2,
                         double theta, double RE, double Pinf, double pV,
                         double sigma, double mu, double rho, double cL,
                         double gamma, double *C)
{
    const double two_pi = 2.0 * M_PI;
    double Pg0 = Pinf - pV + 2.0 * sigma / RE;
    double s = two_pi / (RE * omega1);
    double s2 = s * s;
    C[0] = Pg0 / rho * s2;
    C[1] = (1.0 - 3.0 * gamma) / (rho * cL) * Pg0 * s;
    C[2] = (Pinf - pV) / rho * s2;
    C[3] = 2.0 * sigma / (rho * RE) * s2;
    C[4] = 4.0 * mu / (rho * RE * RE) * (two_pi / omega1);
    C[5] = PA1 / rho * s2;
    C[6] = PA2 / rho * s2;
    C[7] = RE * omega1 * PA1 / (rho * cL) * s2;
    C[8] = RE * omega2 * PA2 / (rho * cL) * s2;
    C[9] = RE * omega1 / (two_pi * cL);
    C[10] = 3.0 * gamma;
    C[11] = omega2 / omega1;
    C[12] = theta;
}
