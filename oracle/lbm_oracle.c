/*
 * Plain FP64 CPU oracle of the 0D-3D coupled lattice Boltzmann time step
 * (arXiv 2112.05258).
 *
 * TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU
 * baseline leg are the only callers.  The product library never links,
 * loads or calls this file, and this file includes nothing from it.
 *
 * It runs Algorithm 1 of the paper step by step, in the paper's order:
 *   1. macroscopic P, v from f (Eqs. rho, v)
 *   2. Lagrangian penalty force B (Eq. LagForce) and Eulerian b (Eq. EulForce)
 *   3. evolve the 0D models one step (Section 2.1.2, forward Euler, Section 2.2)
 *   4. set the boundary populations by non-equilibrium extrapolation
 *      (Eq. Non-equilibrium3)
 *   5. collide (BGK + forcing, Eqs. fi, feq, f) and stream (push form) in Omega,
 *      with halfway bounce-back at rigid walls
 *   6. evolve the wall nodes
 * No loop is fused, blocked or reordered.  Streaming is written in the
 * paper's push form f_i(x + e_i, t + 1) = f*_i(x).
 *
 * Threads: the loops over cells whose iterations write only their own
 * cell's values (macros, force-density reset, forced velocity, collision,
 * streaming) may be spread over orc_set_threads(n) OpenMP threads when the
 * file is compiled with -fopenmp; every reduction, the immersed-boundary
 * spreading and the 0D models stay serial in their fixed order, so the
 * results are the same bits for any thread count.  The default is one
 * thread.
 *
 * Readings of the paper taken where it is silent or ambiguous are stated at
 * the function they affect.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19
#define MAXBC 8

/* threads of the per-cell loops (see the header comment) */
static int g_threads = 1;
#ifdef _OPENMP
#define ORC_PAR_CELLS _Pragma("omp parallel for schedule(static) num_threads(g_threads)")
#else
#define ORC_PAR_CELLS
#endif

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* D3Q19 velocity set: rest, 6 face neighbours, 12 edge neighbours
 * (Section 2.1.1: N_0 = 19, dx/dt = 1). */
static const int EX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
/* Weights of He & Luo's incompressible model (Section 2.1.1). */
static const double W[NQ] = {1.0 / 3,
                             1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

static const double CS2 = 1.0 / 3.0; /* c_s^2 with dx/dt = 1 (Eq. tau) */
static const double RHO0 = 1.0;      /* constant reference density of Eqs. feq, v */
static const double PREF = 1.0 / 3.0; /* lattice pressure at rest: c_s^2 * sum_i w_i */

enum { N_FLUID = 0, N_WALL = 1, N_BC0 = 2 };
enum { BC_VELOCITY = 0, BC_RCR = 1, BC_LV = 2, BC_PRESSURE = 3 };

typedef struct {
    int kind, axis, sign;
    double par[8];
    /* nodes of dOmega_2 belonging to this boundary, raster order */
    long n_nodes;
    long *nodes;
    double *prof; /* n_nodes x 3 (velocity kind) */
    int period;
    double *etab; /* period x 2: E, dE/dt (LV kind) */
    /* links (x_b, i) with x_f = x_b + e_i fluid */
    long n_links;
    long *lk_xb, *lk_xf;
    int *lk_i;
    long *lk_node, *lk_xfi;
    double *lk_ghost;
    /* fluid cells fed by this boundary (the first fluid layer x_f) */
    long n_xf;
    long *xf;
    double *v0; /* n_xf x 3, v(x_f, T_d) for the LV closure */
    /* 0D state */
    double Q, Qu, Pbar;      /* at t_n */
    double Pw, Pv;           /* chamber / ventricle gauge pressure */
    double valve_open, Td;
    double Pstar_gauge;      /* P* - P_ref for pressure-type steps */
} bc_t;

typedef struct {
    int nx, ny, nz;
    long N;
    uint8_t *node;
    double tau;
    int periodic[3];
    int q_scale;
    double *f, *fpost;
    double *P, *jx, *jy, *jz;   /* macroscopic fields at t_n (unforced j) */
    double *vx, *vy, *vz;       /* forced velocity j/rho0 + b/2 */
    double *bx, *by, *bz;       /* Eulerian force density */
    double g[3];                /* uniform external body force (tests only) */
    int nbc;
    bc_t bc[MAXBC];
    /* immersed boundary */
    long ns;
    double *X0, *X, *Vs, *I, *F, *Vf, *dA, *ks;
    uint8_t *pinned;
    double alpha, beta, ms;
    /* filaments (Section 2.3.2's SGFD solid): node lists and (ds, Eh, EI) */
    long n_fil, *fil_start, *fil_count, *fil_nodes;
    double *fil_par, *fil_force;
    long step;
    /* waveform log: one row per step: step, then 4 values per boundary */
    double *wave;
    long wave_rows, wave_cap;
} orc_t;

/* ---------------------------------------------------------------------- */
/* Equations of Section 2.1.1                                              */

/* Eq. feq: incompressible equilibrium (He & Luo). */
void orc_feq(double P, const double v[3], double out[NQ])
{
    double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    for (int i = 0; i < NQ; i++) {
        double ev = EX[i] * v[0] + EY[i] * v[1] + EZ[i] * v[2];
        out[i] = W[i] * P / CS2 +
                 W[i] * RHO0 * (ev / CS2 + ev * ev / (2.0 * CS2 * CS2) - vv / (2.0 * CS2));
    }
}

/* Eq. f: forcing term F_i (Guo form) for velocity v and force density b. */
void orc_forcing(double tau, const double v[3], const double b[3], double out[NQ])
{
    for (int i = 0; i < NQ; i++) {
        double e[3] = {EX[i], EY[i], EZ[i]};
        double ev = e[0] * v[0] + e[1] * v[1] + e[2] * v[2];
        double s = 0.0;
        for (int a = 0; a < 3; a++)
            s += ((e[a] - v[a]) / CS2 + ev / (CS2 * CS2) * e[a]) * b[a];
        out[i] = (1.0 - 1.0 / (2.0 * tau)) * W[i] * s;
    }
}

/* ---------------------------------------------------------------------- */
/* 0D models (Section 2.1.2) and the smoothing of Section 2.2.1            */

/* Eq. SmoothFunction: C-infinity smoothing-to-zero S(t, t0, L_S). */
double orc_smooth(double t, double t0, double LS)
{
    if (t < t0)
        return 1.0;
    if (t > t0 + LS)
        return 0.0;
    double u = (t - t0) / LS;
    if (u <= 0.0)
        return 1.0;
    if (u >= 1.0)
        return 0.0;
    return exp(2.0 * exp(-1.0 / u) / (u - 1.0));
}

/* Eqs. rightbc, rightQ with Z_w = R_p, C_w = C, R_w = R_d, driven by the
 * outflow Q_out: eliminating P between the two equations gives
 *   dP_w/dt = Q_out / C - P_w / (R_d C),   P = P_w + R_p Q_out.
 * One forward-Euler step (dt = 1).  Returns the boundary gauge pressure at
 * t_{n+1} and updates P_w. */
double orc_rcr_step(double *Pw, double Qout, double Rp, double C, double Rd)
{
    double Pw_next = *Pw + (Qout / C - *Pw / (Rd * C));
    *Pw = Pw_next;
    return Pw_next + Rp * Qout;
}

/* Eq. LVE with C_v = 1/E and dC_v/dt = -E'/E^2; one forward-Euler step of
 *   dP_v/dt = -(1/C_v) (dC_v/dt P_v + Q). */
double orc_lv_ode(double Pv, double E, double Edot, double Qin)
{
    double Cv = 1.0 / E;
    double dCv = -Edot / (E * E);
    return Pv - (1.0 / Cv) * (dCv * Pv + Qin);
}

/* Higher-order marching of the same ODEs (the paper allows "forward Euler or
 * higher-order"), with the boundary flow held constant over the step:
 * order 1 forward Euler, 2 Heun (RK2), 4 classical Runge-Kutta. */
static double rcr_rhs(double Pw, double Qout, double C, double Rd) { return Qout / C - Pw / (Rd * C); }

double orc_rcr_step_ord(double *Pw, double Qout, double Rp, double C, double Rd, int order)
{
    double P0 = *Pw, Pn;
    if (order == 2) {
        double k1 = rcr_rhs(P0, Qout, C, Rd);
        double k2 = rcr_rhs(P0 + k1, Qout, C, Rd);
        Pn = P0 + 0.5 * (k1 + k2);
    } else if (order == 4) {
        double k1 = rcr_rhs(P0, Qout, C, Rd);
        double k2 = rcr_rhs(P0 + 0.5 * k1, Qout, C, Rd);
        double k3 = rcr_rhs(P0 + 0.5 * k2, Qout, C, Rd);
        double k4 = rcr_rhs(P0 + k3, Qout, C, Rd);
        Pn = P0 + (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
    } else {
        return orc_rcr_step(Pw, Qout, Rp, C, Rd);
    }
    *Pw = Pn;
    return Pn + Rp * Qout;
}

/* Elastance between table points n and n+1 at s in [0, 1]: cubic Hermite
 * interpolation of (E, dE/dt) at both ends; returns E and writes dE/dt. */
static double hermite_E(double E0, double D0, double E1, double D1, double s, double *dE)
{
    double s2 = s * s, s3 = s2 * s;
    double h00 = 2 * s3 - 3 * s2 + 1, h10 = s3 - 2 * s2 + s, h01 = -2 * s3 + 3 * s2, h11 = s3 - s2;
    double d00 = 6 * s2 - 6 * s, d10 = 3 * s2 - 4 * s + 1, d01 = -6 * s2 + 6 * s, d11 = 3 * s2 - 2 * s;
    *dE = d00 * E0 + d10 * D0 + d01 * E1 + d11 * D1;
    return h00 * E0 + h10 * D0 + h01 * E1 + h11 * D1;
}

/* Eq. LVE as dP_v/dt = (E'/E) P_v - E Q (C_v = 1/E), marched from t_n to
 * t_{n+1} with table values (E0, D0) at t_n and (E1, D1) at t_{n+1}. */
double orc_lv_ode_ord(double Pv, double E0, double D0, double E1, double D1, double Qin, int order)
{
    if (order == 2) {
        double k1 = (D0 / E0) * Pv - E0 * Qin;
        double k2 = (D1 / E1) * (Pv + k1) - E1 * Qin;
        return Pv + 0.5 * (k1 + k2);
    }
    if (order == 4) {
        double Dh, Eh = hermite_E(E0, D0, E1, D1, 0.5, &Dh);
        double k1 = (D0 / E0) * Pv - E0 * Qin;
        double k2 = (Dh / Eh) * (Pv + 0.5 * k1) - Eh * Qin;
        double k3 = (Dh / Eh) * (Pv + 0.5 * k2) - Eh * Qin;
        double k4 = (D1 / E1) * (Pv + k3) - E1 * Qin;
        return Pv + (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
    }
    return orc_lv_ode(Pv, E0, D0, Qin);
}

/* One 0D step of the hybrid LV inlet (Sections 2.1.2, 2.2.1).
 * Inputs: current state, step index n (time t_n), Q_u(t_n), gauge mean
 * boundary pressure at t_n.  Readings:
 *  - the aortic valve opens when the new ventricular gauge pressure exceeds
 *    the mean inlet gauge pressure, and closes when the inflow Q_u < 0; the
 *    close test is not made on the step the valve opened;
 *  - while closed the ventricle refills from an atrial pressure P_la through
 *    an ideal diode (P_v is held at P_la when it would fall below it);
 *  - T_d is t_n of the step at which Q_u < 0 was seen. */
void orc_lv_step_ord(double *Pv, double *valve_open, double *Td, long n,
                     double E, double Edot, double E1, double Edot1, int order,
                     double Qu, double Pbar_gauge, double P_la, int *closed_now)
{
    double Qin = (*valve_open != 0.0) ? Qu : 0.0;
    double Pn = orc_lv_ode_ord(*Pv, E, Edot, E1, Edot1, Qin, order);
    *closed_now = 0;
    if (*valve_open != 0.0) {
        if (Qu < 0.0) {
            *valve_open = 0.0;
            *Td = (double)n;
            *closed_now = 1;
        }
    } else {
        if (Pn < P_la)
            Pn = P_la;
        if (Pn > Pbar_gauge)
            *valve_open = 1.0;
    }
    *Pv = Pn;
}

void orc_lv_step(double *Pv, double *valve_open, double *Td, long n,
                 double E, double Edot, double Qu, double Pbar_gauge,
                 double P_la, int *closed_now)
{
    orc_lv_step_ord(Pv, valve_open, Td, n, E, Edot, E, Edot, 1, Qu, Pbar_gauge, P_la, closed_now);
}

/* ---------------------------------------------------------------------- */
/* Immersed boundary kernel                                                */

/* Discrete delta (reading: 4-point cosine kernel, support |r| < 2). */
double orc_phi(double r)
{
    double a = fabs(r);
    if (a >= 2.0)
        return 0.0;
    return 0.25 * (1.0 + cos(M_PI * r / 2.0));
}

/* ---------------------------------------------------------------------- */

static long cidx(const orc_t *o, int x, int y, int z)
{
    return (long)x + (long)o->nx * ((long)y + (long)o->ny * (long)z);
}

/* neighbour coordinate with optional periodic wrap; returns -1 if outside */
static long nbr(const orc_t *o, int x, int y, int z, int dx, int dy, int dz)
{
    int c[3] = {x + dx, y + dy, z + dz};
    int n[3] = {o->nx, o->ny, o->nz};
    for (int a = 0; a < 3; a++) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (!o->periodic[a])
                return -1;
            c[a] = (c[a] + n[a]) % n[a];
        }
    }
    return cidx(o, c[0], c[1], c[2]);
}

void *orc_create(int nx, int ny, int nz, const uint8_t *node, double tau,
                 int periodic_mask, int q_scale)
{
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    o->nx = nx;
    o->ny = ny;
    o->nz = nz;
    o->N = (long)nx * ny * nz;
    o->tau = tau;
    o->q_scale = q_scale;
    for (int a = 0; a < 3; a++)
        o->periodic[a] = (periodic_mask >> a) & 1;
    o->node = (uint8_t *)malloc(o->N);
    memcpy(o->node, node, o->N);
    o->f = (double *)malloc(sizeof(double) * NQ * o->N);
    o->fpost = (double *)malloc(sizeof(double) * NQ * o->N);
    double **fields[] = {&o->P, &o->jx, &o->jy, &o->jz, &o->vx, &o->vy, &o->vz,
                         &o->bx, &o->by, &o->bz};
    for (int k = 0; k < 10; k++)
        *fields[k] = (double *)calloc(o->N, sizeof(double));
    /* initial state (Section 2.3.2): fluid at rest, P = P_ref */
    for (int i = 0; i < NQ; i++)
        for (long c = 0; c < o->N; c++)
            o->f[i * o->N + c] = W[i];
    return o;
}

/* Registers boundary k (= number of boundaries added so far) and builds its
 * node, link and first-fluid-layer lists.  The first fluid layer x_f of a
 * boundary is read as the set of fluid cells that receive at least one
 * population from one of its nodes (the cells updated by Eq.
 * Non-equilibrium3); its size is the boundary area A in lattice units. */
int orc_add_boundary(void *h, int kind, int axis, int sign, const double *par, int npar,
                     const double *prof, long nprof, const double *etab, int period)
{
    orc_t *o = (orc_t *)h;
    if (o->nbc >= MAXBC)
        return -1;
    int k = o->nbc++;
    bc_t *b = &o->bc[k];
    memset(b, 0, sizeof(*b));
    b->kind = kind;
    b->axis = axis;
    b->sign = sign;
    for (int p = 0; p < npar && p < 8; p++)
        b->par[p] = par[p];
    uint8_t code = (uint8_t)(N_BC0 + k);
    for (long c = 0; c < o->N; c++)
        if (o->node[c] == code)
            b->n_nodes++;
    b->nodes = (long *)malloc(sizeof(long) * (b->n_nodes + 1));
    long m = 0;
    for (long c = 0; c < o->N; c++)
        if (o->node[c] == code)
            b->nodes[m++] = c;
    if (kind == BC_VELOCITY) {
        if (nprof != b->n_nodes)
            return -2;
        b->prof = (double *)malloc(sizeof(double) * 3 * (nprof + 1));
        memcpy(b->prof, prof, sizeof(double) * 3 * nprof);
    }
    if (kind == BC_LV) {
        b->period = period;
        b->etab = (double *)malloc(sizeof(double) * 2 * period);
        memcpy(b->etab, etab, sizeof(double) * 2 * period);
    }
    /* links */
    long cap = b->n_nodes * NQ + 1;
    b->lk_xb = (long *)malloc(sizeof(long) * cap);
    b->lk_xf = (long *)malloc(sizeof(long) * cap);
    b->lk_i = (int *)malloc(sizeof(int) * cap);
    b->lk_node = (long *)malloc(sizeof(long) * cap);
    b->lk_xfi = (long *)malloc(sizeof(long) * cap);
    b->lk_ghost = (double *)malloc(sizeof(double) * cap);
    long *xf_of = (long *)malloc(sizeof(long) * o->N);
    for (long c = 0; c < o->N; c++)
        xf_of[c] = -1;
    b->xf = (long *)malloc(sizeof(long) * cap);
    for (long a = 0; a < b->n_nodes; a++) {
        long c = b->nodes[a];
        int x = (int)(c % o->nx), y = (int)((c / o->nx) % o->ny), z = (int)(c / ((long)o->nx * o->ny));
        for (int i = 1; i < NQ; i++) {
            long t = nbr(o, x, y, z, EX[i], EY[i], EZ[i]);
            if (t < 0 || o->node[t] != N_FLUID)
                continue;
            long L = b->n_links++;
            b->lk_xb[L] = c;
            b->lk_xf[L] = t;
            b->lk_i[L] = i;
            b->lk_node[L] = a;
            if (xf_of[t] < 0) {
                xf_of[t] = b->n_xf;
                b->xf[b->n_xf++] = t;
            }
            b->lk_xfi[L] = xf_of[t];
        }
    }
    free(xf_of);
    b->v0 = (double *)calloc(3 * (b->n_xf + 1), sizeof(double));
    /* initial 0D state (Section 2.3.2: Q_0 = 0) */
    if (kind == BC_RCR)
        b->Pw = b->par[3];
    if (kind == BC_LV) {
        b->Pv = b->par[3];
        b->valve_open = 0.0;
        b->Td = -1e300;
    }
    return k;
}

int orc_set_ib(void *h, long ns, const double *X0, const double *dA, const double *ks,
               const uint8_t *pinned, double alpha, double beta, double ms)
{
    orc_t *o = (orc_t *)h;
    o->ns = ns;
    double **arr3[] = {&o->X0, &o->X, &o->Vs, &o->I, &o->F, &o->Vf};
    for (int k = 0; k < 6; k++)
        *arr3[k] = (double *)calloc(3 * (ns + 1), sizeof(double));
    o->dA = (double *)malloc(sizeof(double) * (ns + 1));
    o->ks = (double *)malloc(sizeof(double) * (ns + 1));
    o->pinned = (uint8_t *)malloc(ns + 1);
    memcpy(o->X0, X0, sizeof(double) * 3 * ns);
    memcpy(o->X, X0, sizeof(double) * 3 * ns);
    memcpy(o->dA, dA, sizeof(double) * ns);
    memcpy(o->ks, ks, sizeof(double) * ns);
    memcpy(o->pinned, pinned, ns);
    o->alpha = alpha;
    o->beta = beta;
    o->ms = ms;
    return 0;
}

/* Overrides the current wall-node positions and velocities (restart, tests). */
void orc_set_ib_state(void *h, const double *X, const double *Vs)
{
    orc_t *o = (orc_t *)h;
    memcpy(o->X, X, sizeof(double) * 3 * o->ns);
    memcpy(o->Vs, Vs, sizeof(double) * 3 * o->ns);
}

/* Declares n_fil filaments over the wall nodes: filament k is the node list
 * nodes[start[k] .. start[k] + count[k] - 1] in arc-length order with
 * par[3k..3k+2] = (ds, Eh, EI).  Its interior nodes move by the SGFD
 * tension and bending forces (orc_filament_force) in addition to the
 * tether spring and the penalty force; its end nodes should be pinned. */
int orc_set_filaments(void *h, long n_fil, const long *start, const long *count, const long *nodes,
                      const double *par)
{
    orc_t *o = (orc_t *)h;
    long tot = 0;
    for (long k = 0; k < n_fil; k++)
        if (start[k] + count[k] > tot)
            tot = start[k] + count[k];
    o->n_fil = n_fil;
    o->fil_start = (long *)malloc(sizeof(long) * (n_fil + 1));
    o->fil_count = (long *)malloc(sizeof(long) * (n_fil + 1));
    o->fil_nodes = (long *)malloc(sizeof(long) * (tot + 1));
    o->fil_par = (double *)malloc(sizeof(double) * 3 * (n_fil + 1));
    o->fil_force = (double *)calloc(3 * (o->ns + 1), sizeof(double));
    memcpy(o->fil_start, start, sizeof(long) * n_fil);
    memcpy(o->fil_count, count, sizeof(long) * n_fil);
    memcpy(o->fil_nodes, nodes, sizeof(long) * tot);
    memcpy(o->fil_par, par, sizeof(double) * 3 * n_fil);
    return 0;
}

/* A uniform body force g (tests only).  It is also, from now until the next
 * step replaces it, the force density b held at every fluid node, so that a
 * read-out taken before the first step (the wall shear stress) sees the b
 * that the step producing the current populations would have used; any
 * immersed-boundary contribution is re-spread by the next step. */
void orc_set_body_force(void *h, double gx, double gy, double gz)
{
    orc_t *o = (orc_t *)h;
    o->g[0] = gx;
    o->g[1] = gy;
    o->g[2] = gz;
    for (long c = 0; c < o->N; c++) {
        int fl = o->node[c] == N_FLUID;
        o->bx[c] = fl ? gx : 0.0;
        o->by[c] = fl ? gy : 0.0;
        o->bz[c] = fl ? gz : 0.0;
    }
}

void orc_set_populations(void *h, const double *f)
{
    orc_t *o = (orc_t *)h;
    memcpy(o->f, f, sizeof(double) * NQ * o->N);
}

void orc_get_populations(void *h, double *f)
{
    orc_t *o = (orc_t *)h;
    memcpy(f, o->f, sizeof(double) * NQ * o->N);
}

/* Sub-step 1 (Eqs. rho, v without the force term): P = c_s^2 sum f,
 * j = sum e f at every fluid node. */
static void compute_macros(orc_t *o)
{
    ORC_PAR_CELLS
    for (long c = 0; c < o->N; c++) {
        o->P[c] = o->jx[c] = o->jy[c] = o->jz[c] = 0.0;
        if (o->node[c] != N_FLUID)
            continue;
        double s = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < NQ; i++) {
            double fi = o->f[i * o->N + c];
            s += fi;
            jx += EX[i] * fi;
            jy += EY[i] * fi;
            jz += EZ[i] * fi;
        }
        o->P[c] = CS2 * s;
        o->jx[c] = jx;
        o->jy[c] = jy;
        o->jz[c] = jz;
    }
}

/* lattice node nearest below X - 0.5 along one axis, and the 4 support
 * cells (i0-1 .. i0+2); returns the cell index or -1 if outside */
static long support_cell(const orc_t *o, int ix, int iy, int iz)
{
    int c[3] = {ix, iy, iz};
    int n[3] = {o->nx, o->ny, o->nz};
    for (int a = 0; a < 3; a++) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (!o->periodic[a])
                return -1;
            c[a] = ((c[a] % n[a]) + n[a]) % n[a];
        }
    }
    return cidx(o, c[0], c[1], c[2]);
}

/* Sub-step 2: penalty force (Eq. LagForce) from the interpolated velocity
 * (Eq. interpolation) and spreading to the lattice (Eq. EulForce).
 * Readings: the interpolated field is the fluid velocity of Eq. v,
 * j/rho0 + b/(2 rho0), formed with the force density b still held from the
 * previous step (the new b depends on V_f, so it cannot enter V_f); the
 * integral is updated before B is formed; the force on the fluid is
 * F = alpha I + beta (V_f - V_s) with alpha, beta < 0 and is spread with a
 * plus sign (the wall receives -F), which makes the penalty a feedback that
 * drives V_f towards V_s.  All nodes interpolate before any node spreads. */
static void ib_force(orc_t *o)
{
    for (long s = 0; s < o->ns; s++) {
        double *X = &o->X[3 * s];
        int i0[3];
        for (int a = 0; a < 3; a++)
            i0[a] = (int)floor(X[a] - 0.5);
        double Vf[3] = {0, 0, 0};
        for (int dz = -1; dz <= 2; dz++)
            for (int dy = -1; dy <= 2; dy++)
                for (int dx = -1; dx <= 2; dx++) {
                    int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                    double d = orc_phi(ix + 0.5 - X[0]) * orc_phi(iy + 0.5 - X[1]) *
                               orc_phi(iz + 0.5 - X[2]);
                    long c = support_cell(o, ix, iy, iz);
                    if (c < 0 || o->node[c] != N_FLUID)
                        continue;
                    Vf[0] += (o->jx[c] + 0.5 * o->bx[c]) / RHO0 * d;
                    Vf[1] += (o->jy[c] + 0.5 * o->by[c]) / RHO0 * d;
                    Vf[2] += (o->jz[c] + 0.5 * o->bz[c]) / RHO0 * d;
                }
        for (int a = 0; a < 3; a++)
            o->Vf[3 * s + a] = Vf[a];
    }
    ORC_PAR_CELLS
    for (long c = 0; c < o->N; c++) {
        int fl = o->node[c] == N_FLUID;
        o->bx[c] = fl ? o->g[0] : 0.0;
        o->by[c] = fl ? o->g[1] : 0.0;
        o->bz[c] = fl ? o->g[2] : 0.0;
    }
    for (long s = 0; s < o->ns; s++) {
        double *X = &o->X[3 * s];
        int i0[3];
        for (int a = 0; a < 3; a++)
            i0[a] = (int)floor(X[a] - 0.5);
        for (int a = 0; a < 3; a++) {
            double dv = o->Vf[3 * s + a] - o->Vs[3 * s + a];
            o->I[3 * s + a] += dv;
            o->F[3 * s + a] = o->alpha * o->I[3 * s + a] + o->beta * dv;
        }
        /* spreading */
        for (int dz = -1; dz <= 2; dz++)
            for (int dy = -1; dy <= 2; dy++)
                for (int dx = -1; dx <= 2; dx++) {
                    int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                    double d = orc_phi(ix + 0.5 - X[0]) * orc_phi(iy + 0.5 - X[1]) *
                               orc_phi(iz + 0.5 - X[2]);
                    long c = support_cell(o, ix, iy, iz);
                    if (c < 0 || o->node[c] != N_FLUID)
                        continue;
                    o->bx[c] += o->F[3 * s + 0] * d * o->dA[s];
                    o->by[c] += o->F[3 * s + 1] * d * o->dA[s];
                    o->bz[c] += o->F[3 * s + 2] * d * o->dA[s];
                }
    }
}

/* Eq. v with dt = 1: v = j/rho0 + b/(2 rho0). */
static void forced_velocity(orc_t *o)
{
    ORC_PAR_CELLS
    for (long c = 0; c < o->N; c++) {
        o->vx[c] = o->jx[c] / RHO0 + o->bx[c] / (2.0 * RHO0);
        o->vy[c] = o->jy[c] / RHO0 + o->by[c] / (2.0 * RHO0);
        o->vz[c] = o->jz[c] / RHO0 + o->bz[c] / (2.0 * RHO0);
    }
}

/* Boundary flow Q(t_n) = sum over x_f of n . (sum e f)/(sum f) with dA = 1
 * (Section 2.1.2), positive into the domain, and the mean pressure over x_f.
 * Q_u = Q / A when q_scale is set (reading: the paper's velocity scale
 * U = Q/A, Section 2.1.4), else Q. */
static void boundary_fluxes(orc_t *o)
{
    for (int k = 0; k < o->nbc; k++) {
        bc_t *b = &o->bc[k];
        double Q = 0.0, Ps = 0.0;
        for (long a = 0; a < b->n_xf; a++) {
            long c = b->xf[a];
            double j[3] = {o->jx[c], o->jy[c], o->jz[c]};
            double sf = o->P[c] / CS2;
            Q += b->sign * j[b->axis] / sf;
            Ps += o->P[c];
        }
        b->Q = Q;
        b->Qu = o->q_scale ? Q / (double)b->n_xf : Q;
        b->Pbar = Ps / (double)b->n_xf;
    }
}

/* Sub-step "evolve ODE to t + dt" for every boundary; sets P* (gauge) for
 * the pressure-type boundaries and records closure velocities. */
static void evolve_0d(orc_t *o)
{
    long n = o->step;
    for (int k = 0; k < o->nbc; k++) {
        bc_t *b = &o->bc[k];
        double Pbar_g = b->Pbar - PREF;
        if (b->kind == BC_RCR) {
            b->Pstar_gauge = orc_rcr_step_ord(&b->Pw, -b->Qu, b->par[0], b->par[1], b->par[2], (int)b->par[4]);
        } else if (b->kind == BC_PRESSURE) {
            b->Pstar_gauge = b->par[0];
        } else if (b->kind == BC_LV) {
            int T = b->period;
            double E = b->etab[2 * (n % T) + 0];
            double Edot = b->etab[2 * (n % T) + 1];
            double E1 = b->etab[2 * ((n + 1) % T) + 0];
            double Edot1 = b->etab[2 * ((n + 1) % T) + 1];
            int closed_now = 0;
            orc_lv_step_ord(&b->Pv, &b->valve_open, &b->Td, n, E, Edot, E1, Edot1, (int)b->par[4],
                            b->Qu, Pbar_g, b->par[1], &closed_now);
            if (closed_now) {
                for (long a = 0; a < b->n_xf; a++) {
                    long c = b->xf[a];
                    b->v0[3 * a + 0] = o->vx[c];
                    b->v0[3 * a + 1] = o->vy[c];
                    b->v0[3 * a + 2] = o->vz[c];
                }
            }
            b->Pstar_gauge = b->Pv;
        }
    }
}

/* Sub-step "couple ODE with LBM on dOmega_2": Eq. Non-equilibrium3 for every
 * link (x_b, i):  f_i(x_f, t_{n+1}) = f^eq_i(P*, v*)
 *      + (1 - 1/tau) (f_i(x_f, t_n) - f^eq_i(P(x_f), v(x_f))) + F_i(x_f, t_n)
 * with (P*, v*) = (P_0D(t_{n+1}), v(x_f, t_n)) for pressure-type and
 * (P(x_f, t_n), v_0D(t_{n+1})) for velocity-type coupling (Section 2.2). */
static void nee_boundary(orc_t *o)
{
    double tn1 = (double)(o->step + 1);
    for (int k = 0; k < o->nbc; k++) {
        bc_t *b = &o->bc[k];
        int pressure_type = (b->kind == BC_RCR || b->kind == BC_PRESSURE ||
                             (b->kind == BC_LV && b->valve_open != 0.0));
        double S = 0.0;
        if (b->kind == BC_LV)
            S = orc_smooth(tn1, b->Td, b->par[2]);
        for (long L = 0; L < b->n_links; L++) {
            long xf = b->lk_xf[L];
            int i = b->lk_i[L];
            double vf[3] = {o->vx[xf], o->vy[xf], o->vz[xf]};
            double bf[3] = {o->bx[xf], o->by[xf], o->bz[xf]};
            double Pf = o->P[xf];
            double Ps, vs[3];
            if (pressure_type) {
                Ps = PREF + b->Pstar_gauge;
                vs[0] = vf[0];
                vs[1] = vf[1];
                vs[2] = vf[2];
            } else {
                Ps = Pf;
                vs[0] = vs[1] = vs[2] = 0.0;
                if (b->kind == BC_VELOCITY) {
                    const double *pr = &b->prof[3 * b->lk_node[L]];
                    double w = b->par[0];
                    double un = pr[0] + pr[1] * cos(w * tn1) - pr[2] * sin(w * tn1);
                    vs[b->axis] = b->sign * un;
                } else { /* LV, valve closed: v_0(T_d) S(t, T_d, N_S dt) */
                    const double *v0 = &b->v0[3 * b->lk_xfi[L]];
                    vs[0] = v0[0] * S;
                    vs[1] = v0[1] * S;
                    vs[2] = v0[2] * S;
                }
            }
            double fs[NQ], ff[NQ], Fi[NQ];
            orc_feq(Ps, vs, fs);
            orc_feq(Pf, vf, ff);
            orc_forcing(o->tau, vf, bf, Fi);
            double fxf = o->f[i * o->N + xf];
            b->lk_ghost[L] = fs[i] + (1.0 - 1.0 / o->tau) * (fxf - ff[i]) + Fi[i];
        }
    }
}

/* Sub-step 3: BGK collision with forcing (Eq. fi) at every fluid node. */
static void collide(orc_t *o)
{
    ORC_PAR_CELLS
    for (long c = 0; c < o->N; c++) {
        if (o->node[c] != N_FLUID)
            continue;
        double v[3] = {o->vx[c], o->vy[c], o->vz[c]};
        double b[3] = {o->bx[c], o->by[c], o->bz[c]};
        double feq[NQ], Fi[NQ];
        orc_feq(o->P[c], v, feq);
        orc_forcing(o->tau, v, b, Fi);
        for (int i = 0; i < NQ; i++) {
            double fi = o->f[i * o->N + c];
            o->fpost[i * o->N + c] = fi - (fi - feq[i]) / o->tau + Fi[i];
        }
    }
}

/* Streaming, push form: f_i(x + e_i, t + 1) = f*_i(x).  A population whose
 * target is a rigid wall (or outside a non-periodic box) returns to x in the
 * opposite direction (halfway bounce-back).  Targets on dOmega_2 are dropped;
 * populations leaving dOmega_2 nodes are the extrapolated ones. */
static void stream(orc_t *o)
{
    static const int OPP[NQ] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
    /* every f_i(t) slot is written by exactly one (cell, direction): a push
     * into a fluid target, or the bounce-back into the own cell */
    ORC_PAR_CELLS
    for (long c = 0; c < o->N; c++) {
        if (o->node[c] != N_FLUID)
            continue;
        int x = (int)(c % o->nx), y = (int)((c / o->nx) % o->ny), z = (int)(c / ((long)o->nx * o->ny));
        for (int i = 0; i < NQ; i++) {
            long t = nbr(o, x, y, z, EX[i], EY[i], EZ[i]);
            double v = o->fpost[i * o->N + c];
            if (t < 0 || o->node[t] == N_WALL)
                o->f[OPP[i] * o->N + c] = v;
            else if (o->node[t] == N_FLUID)
                o->f[i * o->N + t] = v;
        }
    }
    for (int k = 0; k < o->nbc; k++) {
        bc_t *b = &o->bc[k];
        for (long L = 0; L < b->n_links; L++)
            o->f[b->lk_i[L] * o->N + b->lk_xf[L]] = b->lk_ghost[L];
    }
}

/* Internal force per unit reference length of a filament (Section 2.3.2,
 * SGFD): for the nodes X_0 .. X_{n-1} at arc-length spacing ds, with ghost
 * nodes X_{-1} = gl and X_n = gr,
 *   tension  T_{i+1/2} = Eh (|D0 X_{i+1/2}| - 1), D0 X_{i+1/2} = (X_{i+1} - X_i)/ds
 *            (Eq. tension), force (T D0 X)_{i+1/2} - (T D0 X)_{i-1/2}, over ds
 *            (Eq. tension's D0(T D0 X));
 *   bending  -EI D+D-(D+D- X)_i with D+D- X_i = (X_{i+1} - 2 X_i + X_{i-1})/ds^2
 *            (Eqs. 2nd order, bending).
 * out[3i..3i+2] is written for the interior nodes 1 .. n-2 and zeroed at
 * both ends (n >= 3). */
void orc_filament_force(long n, const double *X, const double *gl, const double *gr, double ds, double Eh,
                        double EI, double *out)
{
    double *P = (double *)malloc(sizeof(double) * 3 * (n + 2)); /* X_{-1} .. X_n */
    double *K = (double *)malloc(sizeof(double) * 3 * n);       /* D+D- X_i, i = 0..n-1 */
    double *TD = (double *)malloc(sizeof(double) * 3 * n);      /* (T D0 X)_{i+1/2}, i = 0..n-2 */
    for (int a = 0; a < 3; a++) {
        P[a] = gl[a];
        P[3 * (n + 1) + a] = gr[a];
    }
    memcpy(P + 3, X, sizeof(double) * 3 * n);
    for (long i = 0; i < n; i++)
        for (int a = 0; a < 3; a++)
            K[3 * i + a] = (P[3 * (i + 2) + a] - 2.0 * P[3 * (i + 1) + a] + P[3 * i + a]) / (ds * ds);
    for (long i = 0; i + 1 < n; i++) {
        double d[3], len2 = 0.0;
        for (int a = 0; a < 3; a++) {
            d[a] = (X[3 * (i + 1) + a] - X[3 * i + a]) / ds;
            len2 += d[a] * d[a];
        }
        double T = Eh * (sqrt(len2) - 1.0);
        for (int a = 0; a < 3; a++)
            TD[3 * i + a] = T * d[a];
    }
    for (int a = 0; a < 3; a++)
        out[a] = out[3 * (n - 1) + a] = 0.0;
    for (long i = 1; i + 1 < n; i++)
        for (int a = 0; a < 3; a++) {
            double ten = (TD[3 * i + a] - TD[3 * (i - 1) + a]) / ds;
            double bend = -EI * (K[3 * (i + 1) + a] - 2.0 * K[3 * i + a] + K[3 * (i - 1) + a]) / (ds * ds);
            out[3 * i + a] = ten + bend;
        }
    free(P);
    free(K);
    free(TD);
}

/* Internal forces of every filament at X(t_n), before any node moves.
 * Reading: the wall's filament ends are simply supported (position held,
 * zero curvature), i.e. ghost nodes X_{-1} = 2 X_0 - X_1 and
 * X_n = 2 X_{n-1} - X_{n-2}. */
static void filament_forces(orc_t *o)
{
    for (long k = 0; k < o->n_fil; k++) {
        long n = o->fil_count[k];
        const long *nd = o->fil_nodes + o->fil_start[k];
        double *X = (double *)malloc(sizeof(double) * 3 * n), *out = (double *)malloc(sizeof(double) * 3 * n);
        for (long i = 0; i < n; i++)
            for (int a = 0; a < 3; a++)
                X[3 * i + a] = o->X[3 * nd[i] + a];
        double gl[3], gr[3];
        for (int a = 0; a < 3; a++) {
            gl[a] = 2.0 * X[a] - X[3 + a];
            gr[a] = 2.0 * X[3 * (n - 1) + a] - X[3 * (n - 2) + a];
        }
        orc_filament_force(n, X, gl, gr, o->fil_par[3 * k], o->fil_par[3 * k + 1], o->fil_par[3 * k + 2], out);
        for (long i = 0; i < n; i++)
            for (int a = 0; a < 3; a++)
                o->fil_force[3 * nd[i] + a] = out[3 * i + a];
        free(X);
        free(out);
    }
}

/* Wall-node update (reading: linear springs to X0 replace the shell solver;
 * filament nodes add their SGFD force): m_s dV_s/dt = -k_s (X - X0) + F_fil
 * - F, symplectic Euler with dt = 1 (for a filament this is the central
 * difference in time, X^{n+1} - 2 X^n + X^{n-1} = dt^2 a^n); pinned nodes
 * stay. */
static void solid_update(orc_t *o)
{
    if (o->n_fil)
        filament_forces(o);
    for (long s = 0; s < o->ns; s++) {
        if (o->pinned[s])
            continue;
        for (int a = 0; a < 3; a++) {
            double ff = o->n_fil ? o->fil_force[3 * s + a] : 0.0;
            double acc = (-o->ks[s] * (o->X[3 * s + a] - o->X0[3 * s + a]) + ff - o->F[3 * s + a]) / o->ms;
            o->Vs[3 * s + a] += acc;
            o->X[3 * s + a] += o->Vs[3 * s + a];
        }
    }
}

static void log_wave(orc_t *o)
{
    long width = 1 + 4 * o->nbc;
    if (o->wave_rows + 1 > o->wave_cap) {
        o->wave_cap = o->wave_cap ? 2 * o->wave_cap : 1024;
        o->wave = (double *)realloc(o->wave, sizeof(double) * width * o->wave_cap);
    }
    double *row = &o->wave[o->wave_rows * width];
    row[0] = (double)o->step;
    for (int k = 0; k < o->nbc; k++) {
        bc_t *b = &o->bc[k];
        row[1 + 4 * k + 0] = b->Qu;
        row[1 + 4 * k + 1] = b->Pbar - PREF;
        row[1 + 4 * k + 2] = (b->kind == BC_RCR) ? b->Pw : (b->kind == BC_LV ? b->Pv : b->Pstar_gauge);
        row[1 + 4 * k + 3] = b->valve_open;
    }
    o->wave_rows++;
}

void orc_step(void *h, long nsteps)
{
    orc_t *o = (orc_t *)h;
    for (long s = 0; s < nsteps; s++) {
        compute_macros(o);
        ib_force(o);
        forced_velocity(o);
        boundary_fluxes(o);
        evolve_0d(o);
        nee_boundary(o);
        collide(o);
        stream(o);
        solid_update(o);
        log_wave(o);
        o->step++;
    }
}

/* P = c_s^2 sum f and j = sum e f of the current f(t_n) (no force term). */
void orc_get_macros(void *h, double *P, double *jx, double *jy, double *jz)
{
    orc_t *o = (orc_t *)h;
    compute_macros(o);
    memcpy(P, o->P, sizeof(double) * o->N);
    memcpy(jx, o->jx, sizeof(double) * o->N);
    memcpy(jy, o->jy, sizeof(double) * o->N);
    memcpy(jz, o->jz, sizeof(double) * o->N);
}

void orc_get_force(void *h, double *bx, double *by, double *bz)
{
    orc_t *o = (orc_t *)h;
    memcpy(bx, o->bx, sizeof(double) * o->N);
    memcpy(by, o->by, sizeof(double) * o->N);
    memcpy(bz, o->bz, sizeof(double) * o->N);
}

/* {t_next, Q(t_n), Q_u(t_n), Pbar_gauge(t_n), state (P_w | P_v | P*),
 *  V - V0 = C_v(t_{n+1}) P_v (LV), valve_open, T_d} */
void orc_get_0d(void *h, int k, double *out)
{
    orc_t *o = (orc_t *)h;
    bc_t *b = &o->bc[k];
    out[0] = (double)o->step;
    out[1] = b->Q;
    out[2] = b->Qu;
    out[3] = b->Pbar - PREF;
    out[4] = (b->kind == BC_RCR) ? b->Pw : (b->kind == BC_LV ? b->Pv : b->Pstar_gauge);
    out[5] = 0.0;
    if (b->kind == BC_LV)
        out[5] = b->Pv / b->etab[2 * (o->step % b->period)];
    out[6] = b->valve_open;
    out[7] = b->Td;
}

/* Wall shear stress at the fluid points next to a rigid wall (Section 3.2:
 * WSS = mu dv_1/dx_3 there).  Reading: the viscous stress of the current f(t_n)
 * from its non-equilibrium part, sigma = -(1 - 1/(2 tau)) [sum_i e_i e_i
 * (f_i - f^eq_i(P, v)) + (v b + b v)/2] with v = j/rho0 + b/2 (Guo forcing);
 * the wall normal n is the normalised sum of e_i over the directions whose
 * pull source is a wall (pointing into the fluid); the output is the
 * tangential traction sigma.n - (n.sigma.n) n, 3 values per box cell, zero
 * away from walls.  The force density b is the one of the last step.
 * The (v b + b v)/2 term is what makes a uniformly accelerated fluid (no
 * velocity gradient) carry no stress: its non-equilibrium second moment is
 * exactly -(v b + b v)/2 under the BGK update with Guo forcing (pinned). */
void orc_wall_shear(void *h, double *out)
{
    orc_t *o = (orc_t *)h;
    compute_macros(o);
    memset(out, 0, sizeof(double) * 3 * o->N);
    for (long c = 0; c < o->N; c++) {
        if (o->node[c] != N_FLUID)
            continue;
        int x = (int)(c % o->nx), y = (int)((c / o->nx) % o->ny), z = (int)(c / ((long)o->nx * o->ny));
        double n[3] = {0, 0, 0};
        int walls = 0;
        for (int i = 1; i < NQ; i++) {
            long src = nbr(o, x, y, z, -EX[i], -EY[i], -EZ[i]);
            if (src < 0 || o->node[src] == N_WALL) {
                n[0] += EX[i];
                n[1] += EY[i];
                n[2] += EZ[i];
                walls++;
            }
        }
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (walls == 0 || nn == 0.0)
            continue;
        for (int a = 0; a < 3; a++)
            n[a] /= nn;
        double b[3] = {o->bx[c], o->by[c], o->bz[c]};
        double v[3] = {o->jx[c] / RHO0 + b[0] / (2 * RHO0), o->jy[c] / RHO0 + b[1] / (2 * RHO0),
                       o->jz[c] / RHO0 + b[2] / (2 * RHO0)};
        double feq[NQ];
        orc_feq(o->P[c], v, feq);
        double sig[3][3];
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++) {
                double pi = 0.0;
                for (int i = 0; i < NQ; i++) {
                    int e[3] = {EX[i], EY[i], EZ[i]};
                    pi += e[a] * e[bb] * (o->f[i * o->N + c] - feq[i]);
                }
                sig[a][bb] = -(1.0 - 1.0 / (2.0 * o->tau)) * (pi + 0.5 * (v[a] * b[bb] + b[a] * v[bb]));
            }
        double t[3], tn = 0.0;
        for (int a = 0; a < 3; a++) {
            t[a] = sig[a][0] * n[0] + sig[a][1] * n[1] + sig[a][2] * n[2];
            tn += t[a] * n[a];
        }
        for (int a = 0; a < 3; a++)
            out[3 * c + a] = t[a] - tn * n[a];
    }
}

long orc_wave_rows(void *h) { return ((orc_t *)h)->wave_rows; }

void orc_get_waves(void *h, double *out)
{
    orc_t *o = (orc_t *)h;
    memcpy(out, o->wave, sizeof(double) * (1 + 4 * o->nbc) * o->wave_rows);
}

void orc_get_ib(void *h, double *X, double *Vs, double *F, double *Vf)
{
    orc_t *o = (orc_t *)h;
    memcpy(X, o->X, sizeof(double) * 3 * o->ns);
    memcpy(Vs, o->Vs, sizeof(double) * 3 * o->ns);
    memcpy(F, o->F, sizeof(double) * 3 * o->ns);
    memcpy(Vf, o->Vf, sizeof(double) * 3 * o->ns);
}

long orc_n_xf(void *h, int k) { return ((orc_t *)h)->bc[k].n_xf; }
long orc_n_links(void *h, int k) { return ((orc_t *)h)->bc[k].n_links; }

void orc_destroy(void *h)
{
    orc_t *o = (orc_t *)h;
    if (!o)
        return;
    free(o->node);
    free(o->f);
    free(o->fpost);
    double *fields[] = {o->P, o->jx, o->jy, o->jz, o->vx, o->vy, o->vz, o->bx, o->by, o->bz};
    for (int k = 0; k < 10; k++)
        free(fields[k]);
    for (int k = 0; k < o->nbc; k++) {
        bc_t *b = &o->bc[k];
        free(b->nodes);
        free(b->prof);
        free(b->etab);
        free(b->lk_xb);
        free(b->lk_xf);
        free(b->lk_i);
        free(b->lk_node);
        free(b->lk_xfi);
        free(b->lk_ghost);
        free(b->xf);
        free(b->v0);
    }
    double *ib[] = {o->X0, o->X, o->Vs, o->I, o->F, o->Vf, o->dA, o->ks};
    for (int k = 0; k < 8; k++)
        free(ib[k]);
    free(o->pinned);
    free(o->wave);
    free(o);
}
