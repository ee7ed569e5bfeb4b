/*
 * Plain FP64 CPU oracle for the dual-number 3D space-charge PIC step.
 * TEST INFRASTRUCTURE ONLY: see adpic_oracle.h. This file shares no code
 * with the CUDA library and must never be linked into it.
 *
 * Built with -ffp-contract=off so that every written operation rounds on
 * its own, identically on x86-64 and aarch64.
 */
#include "adpic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact or recommended values */
static const double C_LIGHT = 299792458.0;      /* m/s */
static const double Q_E = 1.602176634e-19;      /* C */
static const double EPS0 = 8.8541878128e-12;    /* F/m */
static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Dual numbers, Sec. 2. A dual is an array D[0..C-1]: D[0] is the     */
/* value, D[k] (k >= 1) the derivative with respect to parameter k.    */
/* ------------------------------------------------------------------ */

typedef double dual[ORC_MAXC];

static void d_const(int C, double v, double* out) {
    out[0] = v;
    for (int k = 1; k < C; ++k) out[k] = 0.0;
}

static void d_copy(int C, const double* f, double* out) {
    for (int k = 0; k < C; ++k) out[k] = f[k];
}

/* Eq. 1: componentwise sum */
static void d_add(int C, const double* f, const double* g, double* out) {
    for (int k = 0; k < C; ++k) out[k] = f[k] + g[k];
}

static void d_sub(int C, const double* f, const double* g, double* out) {
    for (int k = 0; k < C; ++k) out[k] = f[k] - g[k];
}

/* Eq. 2: (f g, g f_k + f g_k) */
static void d_mul(int C, const double* f, const double* g, double* out) {
    double v = f[0] * g[0];
    double t[ORC_MAXC];
    for (int k = 1; k < C; ++k) t[k] = g[0] * f[k] + f[0] * g[k];
    out[0] = v;
    for (int k = 1; k < C; ++k) out[k] = t[k];
}

/* Eq. 3: (f/g, (f_k g - g_k f) / g^2) */
static void d_div(int C, const double* f, const double* g, double* out) {
    double v = f[0] / g[0];
    double g2 = g[0] * g[0];
    double t[ORC_MAXC];
    for (int k = 1; k < C; ++k) t[k] = (f[k] * g[0] - g[k] * f[0]) / g2;
    out[0] = v;
    for (int k = 1; k < C; ++k) out[k] = t[k];
}

/* Eq. 4: h(F) = (h(f), h'(f) f_k), given h(f) and h'(f) */
static void d_fn(int C, const double* f, double h, double hp, double* out) {
    double t[ORC_MAXC];
    for (int k = 1; k < C; ++k) t[k] = hp * f[k];
    out[0] = h;
    for (int k = 1; k < C; ++k) out[k] = t[k];
}

static void d_sqrt(int C, const double* f, double* out) {
    double s = sqrt(f[0]);
    d_fn(C, f, s, 0.5 / s, out);
}
static void d_sin(int C, const double* f, double* out) { d_fn(C, f, sin(f[0]), cos(f[0]), out); }
static void d_cos(int C, const double* f, double* out) { d_fn(C, f, cos(f[0]), -sin(f[0]), out); }
static void d_sinh(int C, const double* f, double* out) { d_fn(C, f, sinh(f[0]), cosh(f[0]), out); }
static void d_cosh(int C, const double* f, double* out) { d_fn(C, f, cosh(f[0]), sinh(f[0]), out); }
static void d_exp(int C, const double* f, double* out) {
    double e = exp(f[0]);
    d_fn(C, f, e, e, out);
}

static void d_log(int C, const double* f, double* out) { d_fn(C, f, log(f[0]), 1.0 / f[0], out); }
static void d_atan(int C, const double* f, double* out) { d_fn(C, f, atan(f[0]), 1.0 / (1.0 + f[0] * f[0]), out); }

/* a constant times a dual: Eq. 2 with g = (a, 0, ..., 0) */
static void d_cmul(int C, double a, const double* f, double* out) {
    dual g;
    d_const(C, a, g);
    d_mul(C, f, g, out);
}

/* an independent variable X_i = (x, 0, .., 1 at slot i+1, ..) (Sec. 2); slot < 0: constant */
static void d_var(int C, double v, int slot, double* out) {
    d_const(C, v, out);
    if (slot >= 0 && slot + 1 < C) out[slot + 1] = 1.0;
}

void orc_dual_op(int op, int C, const double* f, const double* g, double* out) {
    switch (op) {
        case 0: d_add(C, f, g, out); break;
        case 1: d_sub(C, f, g, out); break;
        case 2: d_mul(C, f, g, out); break;
        case 3: d_div(C, f, g, out); break;
        case 4: d_sqrt(C, f, out); break;
        case 5: d_sin(C, f, out); break;
        case 6: d_cos(C, f, out); break;
        case 7: d_sinh(C, f, out); break;
        case 8: d_cosh(C, f, out); break;
        case 9: d_exp(C, f, out); break;
        default: break;
    }
}

/* f = x3 (2 cos(x1/x2) + x1/x2 + e^{x2}) + 2 x4 + sinh(x4) + x5^2, Sec. 3 */
void orc_testfn(const double x[5], double out[6]) {
    const int C = 6;
    dual X[5], q, t, u, v, two, f;
    for (int i = 0; i < 5; ++i) d_var(C, x[i], i, X[i]);
    d_const(C, 2.0, two);
    d_div(C, X[0], X[1], q);      /* x1/x2 */
    d_cos(C, q, t);
    d_mul(C, two, t, t);          /* 2 cos(x1/x2) */
    d_add(C, t, q, t);            /* + x1/x2 */
    d_exp(C, X[1], u);
    d_add(C, t, u, t);            /* + e^{x2} */
    d_mul(C, X[2], t, f);         /* x3 ( ... ) */
    d_mul(C, two, X[3], u);
    d_add(C, f, u, f);            /* + 2 x4 */
    d_sinh(C, X[3], u);
    d_add(C, f, u, f);            /* + sinh(x4) */
    d_mul(C, X[4], X[4], v);
    d_add(C, f, v, f);            /* + x5^2 */
    d_copy(C, f, out);
}

/* ------------------------------------------------------------------ */
/* Physical constants of the reference particle                        */
/* ------------------------------------------------------------------ */

typedef struct {
    double gamma0, beta0, p0, brho, kperp, kz, qm, q;
} consts;

static consts get_consts(const orc_config* cfg) {
    consts k;
    double mass_kg = cfg->mass_eV * Q_E / (C_LIGHT * C_LIGHT);
    k.q = cfg->charge_e * Q_E;
    k.gamma0 = 1.0 + cfg->kinetic_eV / cfg->mass_eV;
    k.beta0 = sqrt(1.0 - 1.0 / (k.gamma0 * k.gamma0));
    k.p0 = k.gamma0 * k.beta0 * mass_kg * C_LIGHT;
    k.brho = k.p0 / k.q;
    double v0 = k.beta0 * C_LIGHT;
    /* transverse: rest-frame E_perp over gamma0 (electric and magnetic
       forces of the co-moving bunch combined); longitudinal: E_z,rest */
    k.kperp = k.q / (k.gamma0 * k.p0 * v0);
    k.kz = k.q / (k.p0 * v0);
    k.qm = cfg->N > 0 ? cfg->bunch_charge_C / (double)cfg->N : 0.0;
    return k;
}

void orc_constants(const orc_config* cfg, double out[8]) {
    consts k = get_consts(cfg);
    out[0] = k.gamma0; out[1] = k.beta0; out[2] = k.p0; out[3] = k.brho;
    out[4] = k.kperp; out[5] = k.kz; out[6] = k.qm; out[7] = k.q;
}

/* The reference-particle constants as duals of the kinetic energy E (slot
   energy_slot): gamma0 = 1 + E / (m c^2), beta0 gamma0 = sqrt(gamma0^2 - 1),
   p0 = beta0 gamma0 m c, B rho = p0 / q, v0 = beta0 c, and the kick constants
   of get_consts. With energy_slot < 0 every derivative part is zero. The
   value parts are those of get_consts (the same numbers as without the slot). */
typedef struct {
    dual gamma0, bg, brho, kperp, kz, g2;
} dconsts;

static int energy_active(const orc_config* cfg) {
    return cfg->energy_slot >= 0 && cfg->energy_slot + 1 < cfg->P + 1;
}

static void get_dconsts(const orc_config* cfg, dconsts* k) {
    const int C = cfg->P + 1;
    const double mass_kg = cfg->mass_eV * Q_E / (C_LIGHT * C_LIGHT);
    const double q = cfg->charge_e * Q_E;
    dual E, t, one, p0, v0, den, qd;
    d_var(C, cfg->kinetic_eV, cfg->energy_slot, E);
    d_const(C, 1.0, one);
    d_cmul(C, 1.0 / cfg->mass_eV, E, t);
    d_add(C, one, t, k->gamma0);
    d_mul(C, k->gamma0, k->gamma0, t);
    d_sub(C, t, one, t);
    d_sqrt(C, t, k->bg);
    d_cmul(C, mass_kg * C_LIGHT, k->bg, p0);
    d_cmul(C, 1.0 / q, p0, k->brho);
    d_div(C, k->bg, k->gamma0, t);
    d_cmul(C, C_LIGHT, t, v0);                 /* v0 = beta0 c */
    d_const(C, q, qd);
    d_mul(C, k->gamma0, p0, den);
    d_mul(C, den, v0, den);
    d_div(C, qd, den, k->kperp);               /* q / (gamma0 p0 v0) */
    d_mul(C, p0, v0, den);
    d_div(C, qd, den, k->kz);                  /* q / (p0 v0) */
    d_mul(C, k->gamma0, k->gamma0, k->g2);
    const consts K = get_consts(cfg);
    k->gamma0[0] = K.gamma0;
    k->bg[0] = K.beta0 * K.gamma0;
    k->brho[0] = K.brho;
    k->kperp[0] = K.kperp;
    k->kz[0] = K.kz;
    k->g2[0] = K.gamma0 * K.gamma0;
}

void orc_dual_constants(const orc_config* cfg, double* out) {
    const int C = cfg->P + 1;
    dconsts k;
    get_dconsts(cfg, &k);
    const double* v[6] = {k.gamma0, k.bg, k.brho, k.kperp, k.kz, k.g2};
    for (int i = 0; i < 6; ++i) d_copy(C, v[i], out + i * C);
}

/* ------------------------------------------------------------------ */
/* Lattice: element of a kick, dual step length, half-step maps         */
/* ------------------------------------------------------------------ */

static int n_elements(const orc_config* cfg) { return cfg->n_line > 0 ? cfg->n_line : 5; }
static int element_kicks(const orc_config* cfg, int e) { return cfg->n_line > 0 ? cfg->line_kicks[e] : cfg->kicks[e]; }

static int kicks_per_period(const orc_config* cfg) {
    int s = 0;
    for (int e = 0; e < n_elements(cfg); ++e) s += element_kicks(cfg, e);
    return s;
}

static int element_of_kick(const orc_config* cfg, int64_t kick) {
    int kpp = kicks_per_period(cfg);
    int s = (int)(kick % kpp);
    for (int e = 0; e < n_elements(cfg); ++e) {
        if (s < element_kicks(cfg, e)) return e;
        s -= element_kicks(cfg, e);
    }
    return n_elements(cfg) - 1;
}

/* parameter index of each element length in lat_slot */
static const int LEN_PARAM[5] = {0, 1, 3, 4, 6};

/* D tau = D L_e / n_e (Sec. 4: step size = element length over the number of steps) */
static void dual_tau(const orc_config* cfg, int e, double* tau) {
    const int C = cfg->P + 1;
    dual L, n;
    if (cfg->n_line > 0) d_var(C, cfg->line[e].L, cfg->line[e].slot_L, L);
    else d_var(C, cfg->L[e], cfg->lat_slot[LEN_PARAM[e]], L);
    d_const(C, (double)element_kicks(cfg, e), n);
    d_div(C, L, n, tau);
}

/* 2x2 dual map of one transverse plane over a step t for focusing strength kp */
static void plane_map(int C, const double* kp, const double* t, double m[4][ORC_MAXC]) {
    dual w, th, c, s, negk;
    if (kp[0] > 0.0) {                 /* focusing plane, Eq. quadtr */
        d_sqrt(C, kp, w);
        d_mul(C, w, t, th);
        d_cos(C, th, c);
        d_sin(C, th, s);
        d_copy(C, c, m[0]);
        d_div(C, s, w, m[1]);
        d_mul(C, w, s, m[2]);
        for (int k = 0; k < C; ++k) m[2][k] = -m[2][k];
        d_copy(C, c, m[3]);
    } else if (kp[0] < 0.0) {          /* defocusing plane */
        for (int k = 0; k < C; ++k) negk[k] = -kp[k];
        d_sqrt(C, negk, w);
        d_mul(C, w, t, th);
        d_cosh(C, th, c);
        d_sinh(C, th, s);
        d_copy(C, c, m[0]);
        d_div(C, s, w, m[1]);
        d_mul(C, w, s, m[2]);
        d_copy(C, c, m[3]);
    } else {                           /* field-free: drift */
        d_const(C, 1.0, m[0]);
        d_copy(C, t, m[1]);
        d_const(C, 0.0, m[2]);
        d_const(C, 1.0, m[3]);
    }
}

/* M1(tau/2) of the element owning this kick: m[plane][entry][C] with
   entries (m11, m12, m21, m22) for planes (x,px), (y,py), (z,delta). */
void orc_half_map(const orc_config* cfg, int64_t kick, double* mflat) {
    const int C = cfg->P + 1;
    dconsts K;
    get_dconsts(cfg, &K);
    int e = element_of_kick(cfg, kick);
    dual tau, t, kx, ky, zero;
    double m[4][ORC_MAXC];
    dual_tau(cfg, e, tau);
    d_cmul(C, 0.5, tau, t);
    d_const(C, 0.0, zero);
    if (cfg->n_line > 0) {
        /* a beamline element: its normalised strength k directly (quadrupoles) */
        if (cfg->line[e].type == 1) d_var(C, cfg->line[e].k, cfg->line[e].slot_k, kx);
        else d_copy(C, zero, kx);
        for (int k = 0; k < C; ++k) ky[k] = -kx[k];
    } else if (e == 1 || e == 3) {
        int gi = (e == 1) ? 0 : 1;
        int gslot = cfg->lat_slot[(e == 1) ? 2 : 5];
        dual g;
        d_var(C, cfg->g[gi], gslot, g);
        d_div(C, g, K.brho, kx);              /* k = q g / p0 = g / Brho (Brho dual in the energy) */
        for (int k = 0; k < C; ++k) ky[k] = -kx[k];
    } else {
        d_copy(C, zero, kx);
        d_copy(C, zero, ky);
    }
    plane_map(C, kx, t, m);
    for (int i = 0; i < 4; ++i) d_copy(C, m[i], mflat + (0 * 4 + i) * C);
    plane_map(C, ky, t, m);
    for (int i = 0; i < 4; ++i) d_copy(C, m[i], mflat + (1 * 4 + i) * C);
    /* longitudinal: z += t delta / gamma0^2 */
    dual tz;
    d_div(C, t, K.g2, tz);
    d_const(C, 1.0, mflat + (2 * 4 + 0) * C);
    d_copy(C, tz, mflat + (2 * 4 + 1) * C);
    d_const(C, 0.0, mflat + (2 * 4 + 2) * C);
    d_const(C, 1.0, mflat + (2 * 4 + 3) * C);
}

static inline double* coord(double* state, int64_t N, int C, int c, int64_t i) {
    return state + ((int64_t)c * N + i) * C;
}
static inline const double* ccoord(const double* state, int64_t N, int C, int c, int64_t i) {
    return state + ((int64_t)c * N + i) * C;
}

void orc_apply_half_map(const orc_config* cfg, double* state, int64_t kick) {
    const int C = cfg->P + 1;
    const int64_t N = cfg->N;
    double m[3 * 4 * ORC_MAXC];
    orc_half_map(cfg, kick, m);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int pl = 0; pl < 3; ++pl) {
            double* u = coord(state, N, C, 2 * pl, i);
            double* p = coord(state, N, C, 2 * pl + 1, i);
            const double* m11 = m + (pl * 4 + 0) * C;
            const double* m12 = m + (pl * 4 + 1) * C;
            const double* m21 = m + (pl * 4 + 2) * C;
            const double* m22 = m + (pl * 4 + 3) * C;
            dual a, b, un, pn;
            d_mul(C, m11, u, a);
            d_mul(C, m12, p, b);
            d_add(C, a, b, un);
            d_mul(C, m21, u, a);
            d_mul(C, m22, p, b);
            d_add(C, a, b, pn);
            d_copy(C, un, u);
            d_copy(C, pn, p);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Initial distribution with Twiss parameters as dual variables         */
/* (Sec. 4: initial distribution parameters may be AD variables)        */
/* ------------------------------------------------------------------ */

int orc_beam_init(const orc_config* cfg, const double* normals, double* state) {
    const int C = cfg->P + 1;
    const int64_t N = cfg->N;
    if (C < 1 || C > ORC_MAXC || N < 0) return -1;
    dconsts K;
    get_dconsts(cfg, &K);
    for (int pl = 0; pl < 3; ++pl) {
        dual al, be, ep, epsn, a, b, t;
        int sa = pl < 2 ? cfg->twiss_slot[3 * pl + 0] : -1;
        int sb = pl < 2 ? cfg->twiss_slot[3 * pl + 1] : -1;
        int se = pl < 2 ? cfg->twiss_slot[3 * pl + 2] : -1;
        d_var(C, cfg->alpha[pl], sa, al);
        d_var(C, cfg->beta[pl], sb, be);
        d_const(C, cfg->eps_n[pl], epsn);
        d_div(C, epsn, K.bg, ep);             /* geometric emittance eps_n / (beta0 gamma0) */
        if (se >= 0) d_var(C, ep[0], se, ep);
        d_mul(C, ep, be, t);
        d_sqrt(C, t, a);                      /* sqrt(eps beta) */
        d_div(C, ep, be, t);
        d_sqrt(C, t, b);                      /* sqrt(eps / beta) */
        const double* n1 = normals + (int64_t)(2 * pl) * N;
        const double* n2 = normals + (int64_t)(2 * pl + 1) * N;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            dual u1, u2, x, p, s;
            d_const(C, n1[i], u1);
            d_const(C, n2[i], u2);
            d_mul(C, a, u1, x);               /* x = sqrt(eps beta) u1 */
            d_mul(C, al, u1, s);
            d_sub(C, u2, s, s);
            d_mul(C, b, s, p);                /* p = sqrt(eps/beta) (u2 - alpha u1) */
            d_copy(C, x, coord(state, N, C, 2 * pl, i));
            d_copy(C, p, coord(state, N, C, 2 * pl + 1, i));
        }
    }
    /* subtract the sample mean of every coordinate (dual) */
    if (N > 0) {
        for (int c = 0; c < 6; ++c) {
            dual sum, mean, invn;
            d_const(C, 0.0, sum);
            for (int64_t i = 0; i < N; ++i) d_add(C, sum, ccoord(state, N, C, c, i), sum);
            d_const(C, (double)N, invn);
            d_div(C, sum, invn, mean);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) {
                double* x = coord(state, N, C, c, i);
                d_sub(C, x, mean, x);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid geometry from the value part (not differentiated)              */
/* ------------------------------------------------------------------ */

int orc_geometry(const orc_config* cfg, const double* state, double* geom) {
    const int C = cfg->P + 1;
    const int64_t N = cfg->N;
    const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
    for (int d = 0; d < 3; ++d) {
        double lo = 0.0, hi = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double v = ccoord(state, N, C, 2 * d, i)[0];
            if (!isfinite(v)) return -5;
            if (i == 0 || v < lo) lo = v;
            if (i == 0 || v > hi) hi = v;
        }
        double w = hi - lo;
        if (!(w > 0.0)) w = 1e-6;
        double h = w / (double)(n[d] - 4);
        geom[d] = lo - 1.5 * h;
        geom[3 + d] = h;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Cloud-in-cell weights (linear shape, two nodes per dimension)        */
/* ------------------------------------------------------------------ */

typedef struct {
    int idx[3];
    double w[3][2][ORC_MAXC];   /* dual weights of the lower/upper node per dimension */
} cic;

static int cic_weights(int C, const double* state, int64_t N, int64_t i, const double* geom,
                       const int n[3], cic* out) {
    for (int d = 0; d < 3; ++d) {
        const double* x = ccoord(state, N, C, 2 * d, i);
        dual o, h, u, f, one;
        if (!isfinite(x[0])) return -5;
        d_const(C, geom[d], o);
        d_const(C, geom[3 + d], h);
        d_sub(C, x, o, u);
        d_div(C, u, h, u);                      /* u = (x - origin) / h */
        double fl = floor(u[0]);
        if (fl < 1.0 || fl > (double)(n[d] - 3)) return -6;
        int id = (int)fl;                       /* floor is not differentiated */
        dual idd;
        d_const(C, (double)id, idd);
        d_sub(C, u, idd, f);                    /* fractional offset in the cell */
        d_const(C, 1.0, one);
        d_sub(C, one, f, out->w[d][0]);
        d_copy(C, f, out->w[d][1]);
        out->idx[d] = id;
    }
    return 0;
}

int orc_deposit(const orc_config* cfg, const double* state, const double* geom, double* rho) {
    const int C = cfg->P + 1;
    const int64_t N = cfg->N;
    const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
    const int64_t nn = (int64_t)n[0] * n[1] * n[2];
    consts K = get_consts(cfg);
    int status = 0;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double* priv = (double*)calloc((size_t)nthreads * C * nn, sizeof(double));
    if (!priv) return -1;
    /* macroparticle charge Q / N, dual in Q when the bunch charge is an AD variable */
    dual Qb, Nd, qmd;
    d_var(C, cfg->bunch_charge_C, cfg->charge_slot, Qb);
    d_const(C, N > 0 ? (double)N : 1.0, Nd);
    d_div(C, Qb, Nd, qmd);
    if (N <= 0) d_const(C, 0.0, qmd);
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* my = priv + (int64_t)tid * C * nn;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            cic w;
            int st = cic_weights(C, state, N, i, geom, n, &w);
            if (st) {
#pragma omp critical
                status = st;
                continue;
            }
            for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        dual W, Q;
                        d_mul(C, w.w[0][a], w.w[1][b], W);
                        d_mul(C, W, w.w[2][c], W);
                        d_mul(C, qmd, W, Q);    /* macroparticle charge times weight (Eq. 2) */
                        int64_t node = ((int64_t)(w.idx[2] + c) * n[1] + (w.idx[1] + b)) * n[0] +
                                       (w.idx[0] + a);
                        for (int k = 0; k < C; ++k) my[(int64_t)k * nn + node] += Q[k];
                    }
        }
    }
    memset(rho, 0, sizeof(double) * C * nn);
    for (int t = 0; t < nthreads; ++t)
        for (int64_t j = 0; j < C * nn; ++j) rho[j] += priv[(int64_t)t * C * nn + j];
    free(priv);
    return status;
}

/* ------------------------------------------------------------------ */
/* Integrated Green's function of the open-boundary Poisson problem    */
/* ------------------------------------------------------------------ */

/* An antiderivative of 1/r: d^3 F / dx dy dz = 1/sqrt(x^2+y^2+z^2). */
static double igf_F(double x, double y, double z) {
    double r = sqrt(x * x + y * y + z * z);
    return y * z * log(x + r) + x * z * log(y + r) + x * y * log(z + r) -
           0.5 * x * x * atan(y * z / (x * r)) - 0.5 * y * y * atan(x * z / (y * r)) -
           0.5 * z * z * atan(x * y / (z * r));
}

double orc_igf(double x, double y, double z, double hx, double hy, double hz) {
    double xs[2] = {x - 0.5 * hx, x + 0.5 * hx};
    double ys[2] = {y - 0.5 * hy, y + 0.5 * hy};
    double zs[2] = {z - 0.5 * hz, z + 0.5 * hz};
    double s = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                double sgn = ((a + b + c) % 2 == 1) ? 1.0 : -1.0;   /* + at the (x2,y2,z2) corner */
                s += sgn * igf_F(xs[a], ys[b], zs[c]);
            }
    return s / (4.0 * PI * EPS0 * hx * hy * hz);
}

/* The antiderivative F of 1/r at (x, y, z) with z a dual number (C = 2):
   Eq. 4 through every elementary function of F. */
static void igf_F_dual(double x, double y, const double* z, double* out) {
    const int C = 2;
    dual X, Y, r, t, u, w, acc, a;
    d_const(C, x, X);
    d_const(C, y, Y);
    d_mul(C, z, z, t);
    d_const(C, x * x + y * y, u);
    d_add(C, t, u, t);
    d_sqrt(C, t, r);                                  /* r */
    d_const(C, 0.0, acc);
    /* y z log(x + r) */
    d_add(C, X, r, t); d_log(C, t, t); d_mul(C, z, t, t); d_cmul(C, y, t, t); d_add(C, acc, t, acc);
    /* x z log(y + r) */
    d_add(C, Y, r, t); d_log(C, t, t); d_mul(C, z, t, t); d_cmul(C, x, t, t); d_add(C, acc, t, acc);
    /* x y log(z + r) */
    d_add(C, z, r, t); d_log(C, t, t); d_cmul(C, x * y, t, t); d_add(C, acc, t, acc);
    /* - x^2/2 atan(y z / (x r)) */
    d_cmul(C, y, z, u); d_cmul(C, x, r, w); d_div(C, u, w, t); d_atan(C, t, t);
    d_cmul(C, -0.5 * x * x, t, t); d_add(C, acc, t, acc);
    /* - y^2/2 atan(x z / (y r)) */
    d_cmul(C, x, z, u); d_cmul(C, y, r, w); d_div(C, u, w, t); d_atan(C, t, t);
    d_cmul(C, -0.5 * y * y, t, t); d_add(C, acc, t, acc);
    /* - z^2/2 atan(x y / (z r)) */
    d_const(C, x * y, u); d_mul(C, z, r, w); d_div(C, u, w, t); d_atan(C, t, t);
    d_mul(C, z, z, a); d_cmul(C, -0.5, a, a); d_mul(C, a, t, t); d_add(C, acc, t, acc);
    d_copy(C, acc, out);
}

void orc_igf_dhz(double x, double y, double kz, double hx, double hy, double hz, double out[2]) {
    const int C = 2;
    dual H, zc, Fv, sum, den, G;
    d_var(C, hz, 0, H);                              /* hz as the variable */
    d_const(C, 0.0, sum);
    const double xs[2] = {x - 0.5 * hx, x + 0.5 * hx};
    const double ys[2] = {y - 0.5 * hy, y + 0.5 * hy};
    const double kc[2] = {kz - 0.5, kz + 0.5};         /* corner z = kc hz */
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                const double sgn = ((a + b + c) % 2 == 1) ? 1.0 : -1.0;
                d_cmul(C, kc[c], H, zc);
                igf_F_dual(xs[a], ys[b], zc, Fv);
                d_cmul(C, sgn, Fv, Fv);
                d_add(C, sum, Fv, sum);
            }
    d_cmul(C, 4.0 * PI * EPS0 * hx * hy, H, den);
    d_div(C, sum, den, G);
    out[0] = G[0];
    out[1] = G[1];
}

/* G on the doubled grid (2nx x 2ny x 2nz), even extension: index i maps to
   offset i for i <= n and i - 2n above. Rest-frame spacings (hx, hy, gamma0 hz). */
void orc_green(const orc_config* cfg, const double* geom, double* G) {
    consts K = get_consts(cfg);
    const int mx = 2 * cfg->nx, my = 2 * cfg->ny, mz = 2 * cfg->nz;
    const double hx = geom[3], hy = geom[4], hz = geom[5] * K.gamma0;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < mz; ++k) {
        int ok = k <= cfg->nz ? k : k - mz;
        for (int j = 0; j < my; ++j) {
            int oj = j <= cfg->ny ? j : j - my;
            for (int i = 0; i < mx; ++i) {
                int oi = i <= cfg->nx ? i : i - mx;
                /* the integral depends on |offset| only; evaluate at |offset| */
                G[((int64_t)k * my + j) * mx + i] =
                    orc_igf(fabs((double)oi) * hx, fabs((double)oj) * hy, fabs((double)ok) * hz, hx, hy, hz);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Radix-2 complex FFT (iterative, bit reversal, unnormalised)          */
/* ------------------------------------------------------------------ */

int orc_fft1d(double* re, double* im, int n, int sign) {
    if (n < 1 || (n & (n - 1))) return -1;
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double ang = sign * 2.0 * PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + k, b = s + k + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] = re[a] + tr; im[a] = im[a] + ti;
            }
        }
    }
    return 0;
}

/* 3D FFT of a complex array [mz][my][mx] (split re/im), along x, then y, then z */
static void fft3d(double* re, double* im, int mx, int my, int mz, int sign) {
#pragma omp parallel
    {
        int mmax = mx > my ? mx : my;
        if (mz > mmax) mmax = mz;
        double* lr = (double*)malloc(sizeof(double) * mmax);
        double* li = (double*)malloc(sizeof(double) * mmax);
#pragma omp for schedule(static)
        for (int64_t line = 0; line < (int64_t)my * mz; ++line) {
            int64_t base = line * mx;
            for (int i = 0; i < mx; ++i) { lr[i] = re[base + i]; li[i] = im[base + i]; }
            orc_fft1d(lr, li, mx, sign);
            for (int i = 0; i < mx; ++i) { re[base + i] = lr[i]; im[base + i] = li[i]; }
        }
#pragma omp for schedule(static)
        for (int64_t line = 0; line < (int64_t)mx * mz; ++line) {
            int64_t k = line / mx, i = line % mx;
            for (int j = 0; j < my; ++j) {
                int64_t a = (k * my + j) * mx + i;
                lr[j] = re[a]; li[j] = im[a];
            }
            orc_fft1d(lr, li, my, sign);
            for (int j = 0; j < my; ++j) {
                int64_t a = (k * my + j) * mx + i;
                re[a] = lr[j]; im[a] = li[j];
            }
        }
#pragma omp for schedule(static)
        for (int64_t line = 0; line < (int64_t)mx * my; ++line) {
            for (int k = 0; k < mz; ++k) {
                int64_t a = (int64_t)k * mx * my + line;
                lr[k] = re[a]; li[k] = im[a];
            }
            orc_fft1d(lr, li, mz, sign);
            for (int k = 0; k < mz; ++k) {
                int64_t a = (int64_t)k * mx * my + line;
                re[a] = lr[k]; im[a] = li[k];
            }
        }
        free(lr);
        free(li);
    }
}

/* dG/dE through the rest-frame spacing hz_r = gamma0 hz: dG/dhz_r (with the
   node offsets k hz_r) times dhz_r/dE = hz / (m c^2) */
void orc_green_denergy(const orc_config* cfg, const double* geom, double* GE) {
    consts K = get_consts(cfg);
    const int mx = 2 * cfg->nx, my = 2 * cfg->ny, mz = 2 * cfg->nz;
    const double hx = geom[3], hy = geom[4], hz = geom[5] * K.gamma0;
    const double dhz = geom[5] / cfg->mass_eV;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < mz; ++k) {
        int ok = k <= cfg->nz ? k : k - mz;
        for (int j = 0; j < my; ++j) {
            int oj = j <= cfg->ny ? j : j - my;
            for (int i = 0; i < mx; ++i) {
                int oi = i <= cfg->nx ? i : i - mx;
                double g[2];
                orc_igf_dhz(fabs((double)oi) * hx, fabs((double)oj) * hy, fabs((double)ok), hx, hy, hz, g);
                GE[((int64_t)k * my + j) * mx + i] = g[1] * dhz;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Hockney convolution phi_c = G * rho_c for every channel (Sec. 4: the  */
/* Poisson equation is solved for the value and for every derivative)   */
/* ------------------------------------------------------------------ */

int orc_solve(const orc_config* cfg, const double* geom, const double* rho, double* phi) {
    const int C = cfg->P + 1;
    const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
    const int mx = 2 * nx, my = 2 * ny, mz = 2 * nz;
    const int64_t M = (int64_t)mx * my * mz, nn = (int64_t)nx * ny * nz;
    /* with the kinetic energy as a dual input G is dual too: the energy
       channel gets phi_E = G * rho_E + (dG/dE) * rho_0 (Eq. 2 on the product
       inside the convolution) */
    const int ce = energy_active(cfg) ? cfg->energy_slot + 1 : -1;
    double* gr = (double*)malloc(sizeof(double) * M);
    double* gi = (double*)calloc(M, sizeof(double));
    double* ar = (double*)malloc(sizeof(double) * M);
    double* ai = (double*)malloc(sizeof(double) * M);
    double* er = ce > 0 ? (double*)malloc(sizeof(double) * M) : NULL;
    double* ei = ce > 0 ? (double*)calloc(M, sizeof(double)) : NULL;
    double* r0r = ce > 0 ? (double*)malloc(sizeof(double) * M) : NULL;
    double* r0i = ce > 0 ? (double*)malloc(sizeof(double) * M) : NULL;
    if (!gr || !gi || !ar || !ai || (ce > 0 && (!er || !ei || !r0r || !r0i))) {
        free(gr); free(gi); free(ar); free(ai); free(er); free(ei); free(r0r); free(r0i);
        return -1;
    }
    orc_green(cfg, geom, gr);
    fft3d(gr, gi, mx, my, mz, -1);
    if (ce > 0) {
        orc_green_denergy(cfg, geom, er);
        fft3d(er, ei, mx, my, mz, -1);
    }
    for (int c = 0; c < C; ++c) {
        memset(ar, 0, sizeof(double) * M);
        memset(ai, 0, sizeof(double) * M);
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    ar[((int64_t)k * my + j) * mx + i] = rho[(int64_t)c * nn + ((int64_t)k * ny + j) * nx + i];
        fft3d(ar, ai, mx, my, mz, -1);
        if (c == 0 && ce > 0) {
            memcpy(r0r, ar, sizeof(double) * M);
            memcpy(r0i, ai, sizeof(double) * M);
        }
        for (int64_t q = 0; q < M; ++q) {
            double r = ar[q] * gr[q] - ai[q] * gi[q];
            double s = ar[q] * gi[q] + ai[q] * gr[q];
            if (c == ce) {
                r += r0r[q] * er[q] - r0i[q] * ei[q];
                s += r0r[q] * ei[q] + r0i[q] * er[q];
            }
            ar[q] = r;
            ai[q] = s;
        }
        fft3d(ar, ai, mx, my, mz, +1);
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    phi[(int64_t)c * nn + ((int64_t)k * ny + j) * nx + i] =
                        ar[((int64_t)k * my + j) * mx + i] / (double)M;
    }
    free(gr); free(gi); free(ar); free(ai); free(er); free(ei); free(r0r); free(r0i);
    return 0;
}

/* brute-force direct sum phi_c(i) = sum_j rho_c(j) G(i - j) (pins the FFT path) */
int orc_solve_direct(const orc_config* cfg, const double* geom, const double* rho, double* phi) {
    const int C = cfg->P + 1;
    const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
    const int64_t nn = (int64_t)nx * ny * nz;
    consts K = get_consts(cfg);
    const double hx = geom[3], hy = geom[4], hz = geom[5] * K.gamma0;
    const int ce = energy_active(cfg) ? cfg->energy_slot + 1 : -1;
    const double dhz = geom[5] / cfg->mass_eV;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nn; ++a) {
        int ia = (int)(a % nx), ja = (int)((a / nx) % ny), ka = (int)(a / ((int64_t)nx * ny));
        for (int c = 0; c < C; ++c) phi[(int64_t)c * nn + a] = 0.0;
        for (int64_t b = 0; b < nn; ++b) {
            int ib = (int)(b % nx), jb = (int)((b / nx) % ny), kb = (int)(b / ((int64_t)nx * ny));
            double G = orc_igf(fabs((double)(ia - ib)) * hx, fabs((double)(ja - jb)) * hy,
                               fabs((double)(ka - kb)) * hz, hx, hy, hz);
            for (int c = 0; c < C; ++c) phi[(int64_t)c * nn + a] += G * rho[(int64_t)c * nn + b];
            if (ce > 0) {
                double g[2];
                orc_igf_dhz(fabs((double)(ia - ib)) * hx, fabs((double)(ja - jb)) * hy, fabs((double)(ka - kb)),
                            hx, hy, hz, g);
                phi[(int64_t)ce * nn + a] += g[1] * dhz * rho[b];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Central finite-difference field E = -grad(phi), rest-frame spacing  */
/* ------------------------------------------------------------------ */

void orc_field(const orc_config* cfg, const double* geom, const double* phi, double* E) {
    const int C = cfg->P + 1;
    const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
    const int64_t nn = (int64_t)nx * ny * nz;
    consts K = get_consts(cfg);
    const double hx = geom[3], hy = geom[4], hz = geom[5] * K.gamma0;
    memset(E, 0, sizeof(double) * 3 * C * nn);
    for (int c = 0; c < C; ++c) {
        const double* f = phi + (int64_t)c * nn;
        double* ex = E + ((int64_t)0 * C + c) * nn;
        double* ey = E + ((int64_t)1 * C + c) * nn;
        double* ez = E + ((int64_t)2 * C + c) * nn;
        for (int k = 1; k < nz - 1; ++k)
            for (int j = 1; j < ny - 1; ++j)
                for (int i = 1; i < nx - 1; ++i) {
                    int64_t a = ((int64_t)k * ny + j) * nx + i;
                    ex[a] = -(f[a + 1] - f[a - 1]) / (2.0 * hx);
                    ey[a] = -(f[a + nx] - f[a - nx]) / (2.0 * hy);
                    ez[a] = -(f[a + (int64_t)nx * ny] - f[a - (int64_t)nx * ny]) / (2.0 * hz);
                }
    }
    if (energy_active(cfg)) {
        /* the rest-frame spacing 2 gamma0 hz is dual in the energy: E_z is the
           dual quotient (Eq. 3) of -(phi(k+1) - phi(k-1)) by it */
        dconsts D;
        get_dconsts(cfg, &D);
        dual den;
        d_cmul(C, 2.0 * geom[5], D.gamma0, den);
        for (int k = 1; k < nz - 1; ++k)
            for (int j = 1; j < ny - 1; ++j)
                for (int i = 1; i < nx - 1; ++i) {
                    const int64_t a = ((int64_t)k * ny + j) * nx + i;
                    dual num, q;
                    for (int c = 0; c < C; ++c) {
                        const double* f = phi + (int64_t)c * nn;
                        num[c] = -(f[a + (int64_t)nx * ny] - f[a - (int64_t)nx * ny]);
                    }
                    d_div(C, num, den, q);
                    for (int c = 0; c < C; ++c) E[((int64_t)2 * C + c) * nn + a] = q[c];
                }
    }
}

/* ------------------------------------------------------------------ */
/* Gather (same linear shape as the deposit) and the space-charge kick  */
/* M2(tau): r fixed, p += kappa tau E (Sec. 4, Eqs. for map M2)         */
/* ------------------------------------------------------------------ */

int orc_gather(const orc_config* cfg, const double* state, const double* geom, const double* E,
               double* Ep) {
    const int C = cfg->P + 1;
    const int64_t N = cfg->N;
    const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
    const int64_t nn = (int64_t)n[0] * n[1] * n[2];
    int status = 0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        cic w;
        int st = cic_weights(C, state, N, i, geom, n, &w);
        if (st) {
#pragma omp critical
            status = st;
            continue;
        }
        for (int d = 0; d < 3; ++d) {
            dual acc, W, En, t;
            d_const(C, 0.0, acc);
            for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        d_mul(C, w.w[0][a], w.w[1][b], W);
                        d_mul(C, W, w.w[2][c], W);
                        int64_t node = ((int64_t)(w.idx[2] + c) * n[1] + (w.idx[1] + b)) * n[0] +
                                       (w.idx[0] + a);
                        for (int k = 0; k < C; ++k) En[k] = E[((int64_t)d * C + k) * nn + node];
                        d_mul(C, W, En, t);
                        d_add(C, acc, t, acc);
                    }
            d_copy(C, acc, Ep + ((int64_t)d * N + i) * C);
        }
    }
    return status;
}

int orc_kick(const orc_config* cfg, double* state, const double* geom, const double* E, int64_t kick) {
    const int C = cfg->P + 1;
    const int64_t N = cfg->N;
    dconsts K;
    get_dconsts(cfg, &K);
    double* Ep = (double*)malloc(sizeof(double) * 3 * N * C + 8);
    if (!Ep) return -1;
    int st = orc_gather(cfg, state, geom, E, Ep);
    if (st) { free(Ep); return st; }
    dual tau, a[3];
    dual_tau(cfg, element_of_kick(cfg, kick), tau);
    d_mul(C, tau, K.kperp, a[0]);        /* kappa tau, dual in the step and the energy */
    d_mul(C, tau, K.kperp, a[1]);
    d_mul(C, tau, K.kz, a[2]);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int d = 0; d < 3; ++d) {
            dual dp;
            double* p = coord(state, N, C, 2 * d + 1, i);
            d_mul(C, a[d], Ep + ((int64_t)d * N + i) * C, dp);
            d_add(C, p, dp, p);
        }
    }
    free(Ep);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dual beam moments and emittance (Sec. 4, D eps_x)                    */
/* ------------------------------------------------------------------ */

/* Neumaier's compensated summation (the Kahan-Babuska improvement of Kahan's
   method): *s holds the running sum and *c the accumulated rounding errors, so
   s + c is the sum up to about one rounding, whatever the order of the terms. */
static void nsum_add(double* s, double* c, double x) {
    const double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}

/* Dual moments <u>, <p>, <u^2>, <u p>, <p^2> per plane (Sec. 4, the means of
   the dual emittance), each an average over particles. The emittance
   derivatives cancel strongly (the emittance barely changes while the second
   moments do), so the sums are compensated: their rounding does not depend
   on the summation order (thread count) at the level the derivatives need. */
void orc_moments(const orc_config* cfg, const double* state, double* mom) {
    const int C = cfg->P + 1;
    const int64_t N = cfg->N;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    /* per thread: [5][ORC_MAXC] sums then [5][ORC_MAXC] compensations */
    double* part = (double*)malloc(sizeof(double) * nthreads * 10 * ORC_MAXC);
    for (int pl = 0; pl < 3; ++pl) {
#pragma omp parallel
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            double* t = part + (int64_t)tid * 10 * ORC_MAXC;
            double* tc = t + 5 * ORC_MAXC;
            dual a;
            for (int j = 0; j < 10 * ORC_MAXC; ++j) t[j] = 0.0;
#pragma omp for schedule(static)
            for (int64_t i = 0; i < N; ++i) {
                const double* u = ccoord(state, N, C, 2 * pl, i);
                const double* p = ccoord(state, N, C, 2 * pl + 1, i);
                for (int k = 0; k < C; ++k) {
                    nsum_add(t + 0 * ORC_MAXC + k, tc + 0 * ORC_MAXC + k, u[k]);
                    nsum_add(t + 1 * ORC_MAXC + k, tc + 1 * ORC_MAXC + k, p[k]);
                }
                d_mul(C, u, u, a);
                for (int k = 0; k < C; ++k) nsum_add(t + 2 * ORC_MAXC + k, tc + 2 * ORC_MAXC + k, a[k]);
                d_mul(C, u, p, a);
                for (int k = 0; k < C; ++k) nsum_add(t + 3 * ORC_MAXC + k, tc + 3 * ORC_MAXC + k, a[k]);
                d_mul(C, p, p, a);
                for (int k = 0; k < C; ++k) nsum_add(t + 4 * ORC_MAXC + k, tc + 4 * ORC_MAXC + k, a[k]);
            }
        }
        /* thread partials (sums and compensations) combined in thread order */
        for (int q = 0; q < 5; ++q) {
            dual sq, nd;
            for (int k = 0; k < C; ++k) {
                double s = 0.0, c = 0.0;
                for (int th = 0; th < nthreads; ++th) {
                    const double* t = part + (int64_t)th * 10 * ORC_MAXC;
                    nsum_add(&s, &c, t[q * ORC_MAXC + k]);
                    nsum_add(&s, &c, t[(5 + q) * ORC_MAXC + k]);
                }
                sq[k] = s + c;
            }
            d_const(C, N > 0 ? (double)N : 1.0, nd);
            d_div(C, sq, nd, mom + (pl * 5 + q) * C);
        }
    }
    free(part);
}

void orc_emittance(const orc_config* cfg, const double* mom, double* eps) {
    const int C = cfg->P + 1;
    for (int pl = 0; pl < 3; ++pl) {
        const double* mu = mom + (pl * 5 + 0) * C;
        const double* mp = mom + (pl * 5 + 1) * C;
        const double* uu = mom + (pl * 5 + 2) * C;
        const double* up = mom + (pl * 5 + 3) * C;
        const double* pp = mom + (pl * 5 + 4) * C;
        dual a, b, c, t, d;
        d_mul(C, mu, mu, t); d_sub(C, uu, t, a);     /* centred <u^2> */
        d_mul(C, mu, mp, t); d_sub(C, up, t, b);     /* centred <u p> */
        d_mul(C, mp, mp, t); d_sub(C, pp, t, c);     /* centred <p^2> */
        d_mul(C, a, c, t);
        d_mul(C, b, b, d);
        d_sub(C, t, d, t);
        d_sqrt(C, t, eps + pl * C);
    }
}

/* ------------------------------------------------------------------ */
/* The split-operator run                                               */
/* ------------------------------------------------------------------ */

int orc_run(const orc_config* cfg, double* state, int64_t kick0, int n_kicks, double* mom_hist,
            double* geom_io, int geom_mode) {
    const int C = cfg->P + 1;
    if (C < 1 || C > ORC_MAXC || n_kicks < 0) return -1;
    const int64_t nn = (int64_t)cfg->nx * cfg->ny * cfg->nz;
    const int kpp = kicks_per_period(cfg);
    double* rho = (double*)malloc(sizeof(double) * C * nn);
    double* phi = (double*)malloc(sizeof(double) * C * nn);
    double* E = (double*)malloc(sizeof(double) * 3 * C * nn);
    if (!rho || !phi || !E) { free(rho); free(phi); free(E); return -1; }
    int rec = 0, st = 0;
    for (int s = 0; s < n_kicks; ++s) {
        int64_t kick = kick0 + s;
        double geom[6];
        orc_apply_half_map(cfg, state, kick);             /* M1(tau/2) */
        if (geom_mode == 2) {
            memcpy(geom, geom_io + 6 * s, sizeof(geom));
        } else {
            st = orc_geometry(cfg, state, geom);
            if (st) break;
            if (geom_mode == 1) memcpy(geom_io + 6 * s, geom, sizeof(geom));
        }
        st = orc_deposit(cfg, state, geom, rho);          /* D rho */
        if (st) break;
        st = orc_solve(cfg, geom, rho, phi);              /* D phi */
        if (st) break;
        orc_field(cfg, geom, phi, E);                     /* D E */
        st = orc_kick(cfg, state, geom, E, kick);         /* M2(tau) */
        if (st) break;
        orc_apply_half_map(cfg, state, kick);             /* M1(tau/2) */
        if (((kick + 1) % kpp == 0) || s == n_kicks - 1) {
            if (mom_hist) orc_moments(cfg, state, mom_hist + (int64_t)rec * 15 * C);
            ++rec;
        }
    }
    free(rho); free(phi); free(E);
    return st ? st : rec;
}

/* ------------------------------------------------------------------ */
/* Single-particle dual optics (Sec. 3): transfer matrices of a beamline */
/* of drifts and thick quadrupoles, Twiss transport (Eq. 5), periodic    */
/* Twiss functions of a cell, and element-by-element particle tracking. */
/* ------------------------------------------------------------------ */

/* element map of one plane: quad strength +k in x, -k in y, over length L (Eq. quadtr) */
static void element_plane_map(int C, const orc_element* e, int plane, double m[4][ORC_MAXC]) {
    dual L, k;
    d_var(C, e->L, e->slot_L, L);
    d_var(C, e->type == 1 ? e->k : 0.0, e->type == 1 ? e->slot_k : -1, k);
    if (plane == 1)
        for (int j = 0; j < C; ++j) k[j] = -k[j];
    plane_map(C, k, L, m);
}

/* B A for dual 2x2 matrices (A first along the beam) */
static void mat_mul2(int C, double b[4][ORC_MAXC], double a[4][ORC_MAXC], double out[4][ORC_MAXC]) {
    dual t1, t2, r[4];
    d_mul(C, b[0], a[0], t1); d_mul(C, b[1], a[2], t2); d_add(C, t1, t2, r[0]);
    d_mul(C, b[0], a[1], t1); d_mul(C, b[1], a[3], t2); d_add(C, t1, t2, r[1]);
    d_mul(C, b[2], a[0], t1); d_mul(C, b[3], a[2], t2); d_add(C, t1, t2, r[2]);
    d_mul(C, b[2], a[1], t1); d_mul(C, b[3], a[3], t2); d_add(C, t1, t2, r[3]);
    for (int i = 0; i < 4; ++i) d_copy(C, r[i], out[i]);
}

void orc_beamline_matrix(int P, const orc_element* el, int n, double* m) {
    const int C = P + 1;
    for (int pl = 0; pl < 2; ++pl) {
        double acc[4][ORC_MAXC], em[4][ORC_MAXC];
        d_const(C, 1.0, acc[0]); d_const(C, 0.0, acc[1]); d_const(C, 0.0, acc[2]); d_const(C, 1.0, acc[3]);
        for (int i = 0; i < n; ++i) {
            element_plane_map(C, &el[i], pl, em);
            mat_mul2(C, em, acc, acc);
        }
        for (int j = 0; j < 4; ++j) d_copy(C, acc[j], m + (pl * 4 + j) * C);
    }
}

/* Eq. 5: (beta, alpha) at s from (beta0, alpha0, gamma0) at 0 and the matrix m from 0 to s */
static void twiss_transport(int C, double m[4][ORC_MAXC], const double* b0, const double* a0, double* b, double* a) {
    dual one, g0, t, u, v;
    d_const(C, 1.0, one);
    d_mul(C, a0, a0, t);
    d_add(C, one, t, t);
    d_div(C, t, b0, g0);                                  /* gamma0 = (1 + alpha0^2) / beta0 */
    /* beta = m11^2 beta0 - 2 m11 m12 alpha0 + m12^2 gamma0 */
    d_mul(C, m[0], m[0], t); d_mul(C, t, b0, u);
    d_mul(C, m[0], m[1], t); d_mul(C, t, a0, t); d_cmul(C, 2.0, t, t); d_sub(C, u, t, u);
    d_mul(C, m[1], m[1], t); d_mul(C, t, g0, t); d_add(C, u, t, v);
    d_copy(C, v, b);
    /* alpha = -m11 m21 beta0 + (m11 m22 + m12 m21) alpha0 - m12 m22 gamma0 */
    d_mul(C, m[0], m[2], t); d_mul(C, t, b0, u);
    for (int k = 0; k < C; ++k) u[k] = -u[k];
    d_mul(C, m[0], m[3], t); d_mul(C, m[1], m[2], v); d_add(C, t, v, t); d_mul(C, t, a0, t); d_add(C, u, t, u);
    d_mul(C, m[1], m[3], t); d_mul(C, t, g0, t); d_sub(C, u, t, u);
    d_copy(C, u, a);
}

void orc_twiss(int P, const orc_element* el, int n, const double* twiss0, double* out) {
    const int C = P + 1;
    double m[2 * 4 * ORC_MAXC];
    orc_beamline_matrix(P, el, n, m);
    for (int pl = 0; pl < 2; ++pl) {
        double mm[4][ORC_MAXC];
        dual b0, a0;
        for (int j = 0; j < 4; ++j) d_copy(C, m + (pl * 4 + j) * C, mm[j]);
        d_const(C, twiss0[2 * pl], b0);
        d_const(C, twiss0[2 * pl + 1], a0);
        twiss_transport(C, mm, b0, a0, out + (2 * pl) * C, out + (2 * pl + 1) * C);
    }
}

/* periodic solution of the cell: cos mu = (m11 + m22) / 2, sin mu with the sign of m12,
   beta = m12 / sin mu, alpha = (m11 - m22) / (2 sin mu) */
int orc_periodic_twiss(int P, const orc_element* el, int n, double* out) {
    const int C = P + 1;
    double m[2 * 4 * ORC_MAXC];
    orc_beamline_matrix(P, el, n, m);
    for (int pl = 0; pl < 2; ++pl) {
        const double* m11 = m + (pl * 4 + 0) * C;
        const double* m12 = m + (pl * 4 + 1) * C;
        const double* m22 = m + (pl * 4 + 3) * C;
        dual cs, t, one, s;
        d_add(C, m11, m22, t);
        d_cmul(C, 0.5, t, cs);
        if (!(fabs(cs[0]) < 1.0)) return -1;               /* unstable cell */
        d_const(C, 1.0, one);
        d_mul(C, cs, cs, t);
        d_sub(C, one, t, t);
        d_sqrt(C, t, s);
        if (m12[0] < 0.0)
            for (int k = 0; k < C; ++k) s[k] = -s[k];
        d_div(C, m12, s, out + (2 * pl) * C);
        d_sub(C, m11, m22, t);
        d_cmul(C, 0.5, t, t);
        d_div(C, t, s, out + (2 * pl + 1) * C);
    }
    return 0;
}

void orc_track(int P, const orc_element* el, int n, int64_t n_repeat, int64_t N, const double* x0, double* out) {
    const int C = P + 1;
    /* the element maps do not change from turn to turn */
    double* maps = (double*)malloc(sizeof(double) * (size_t)n * 2 * 4 * ORC_MAXC);
    for (int i = 0; i < n; ++i)
        for (int pl = 0; pl < 2; ++pl) element_plane_map(C, &el[i], pl, (double(*)[ORC_MAXC])(maps + ((size_t)i * 2 + pl) * 4 * ORC_MAXC));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        dual z[4], t1, t2, nx, np;
        for (int c = 0; c < 4; ++c) d_const(C, x0[p * 4 + c], z[c]);
        for (int64_t r = 0; r < n_repeat; ++r)
            for (int i = 0; i < n; ++i)
                for (int pl = 0; pl < 2; ++pl) {
                    double(*mm)[ORC_MAXC] = (double(*)[ORC_MAXC])(maps + ((size_t)i * 2 + pl) * 4 * ORC_MAXC);
                    d_mul(C, mm[0], z[2 * pl], t1); d_mul(C, mm[1], z[2 * pl + 1], t2); d_add(C, t1, t2, nx);
                    d_mul(C, mm[2], z[2 * pl], t1); d_mul(C, mm[3], z[2 * pl + 1], t2); d_add(C, t1, t2, np);
                    d_copy(C, nx, z[2 * pl]);
                    d_copy(C, np, z[2 * pl + 1]);
                }
        for (int c = 0; c < 4; ++c) d_copy(C, z[c], out + (p * 4 + c) * C);
    }
    free(maps);
}

/* ------------------------------------------------------------------ */
/* 2D PIC in a rectangular conducting pipe (Sec. 4): bilinear deposit, */
/* sine-transform Poisson solve, central-difference field, the kick of */
/* H2 = K phi / 2, and the same quadrupole maps in x and y.            */
/* ------------------------------------------------------------------ */

/* derived 2D constants: gamma0, beta0, p0, B rho, the paper's perveance K,
   the kick factor 2 pi K (phi normalised to unit charge, see orc2d_solve) */
static void consts2d(const orc2d_config* c, double* gamma0, double* beta0, double* p0, double* brho, double* K) {
    const double mass_kg = c->mass_eV * Q_E / (C_LIGHT * C_LIGHT);
    const double q = c->charge_e * Q_E;
    *gamma0 = 1.0 + c->kinetic_eV / c->mass_eV;
    *beta0 = sqrt(1.0 - 1.0 / (*gamma0 * *gamma0));
    *p0 = *gamma0 * *beta0 * mass_kg * C_LIGHT;
    *brho = *p0 / q;
    const double v0 = *beta0 * C_LIGHT;
    *K = q * c->current_A / (2.0 * PI * EPS0 * *p0 * v0 * v0 * *gamma0 * *gamma0);
}

void orc2d_constants(const orc2d_config* c, double out[5]) {
    consts2d(c, &out[0], &out[1], &out[2], &out[3], &out[4]);
}

/* the FODO config viewed as a 3D config for the shared map code (half maps only) */
static orc_config as3d(const orc2d_config* c) {
    orc_config k;
    memset(&k, 0, sizeof(k));
    k.P = c->P;
    k.kinetic_eV = c->kinetic_eV;
    k.mass_eV = c->mass_eV;
    k.charge_e = c->charge_e;
    for (int e = 0; e < 5; ++e) { k.L[e] = c->L[e]; k.kicks[e] = c->kicks[e]; }
    k.g[0] = c->g[0];
    k.g[1] = c->g[1];
    for (int j = 0; j < 7; ++j) k.lat_slot[j] = c->lat_slot[j];
    k.charge_slot = -1;
    k.energy_slot = -1;
    return k;
}

/* bilinear weights of particle i: pipe coordinates u = (x + a/2) / hx etc.
   (the beam axis is the pipe centre); cells [0, n-1]; a particle closer
   than one cell to a wall is outside the stencil range */
static int bilinear(int C, const double* state, int64_t N, int64_t i, const orc2d_config* c, int idx[2],
                    double w[2][2][ORC_MAXC]) {
    const double hx = c->a / c->nx, hy = c->b / c->ny;
    const double h[2] = {hx, hy}, off[2] = {0.5 * c->a, 0.5 * c->b};
    const int n[2] = {c->nx, c->ny};
    for (int d = 0; d < 2; ++d) {
        const double* x = state + ((int64_t)(2 * d) * N + i) * C;
        const double u = (x[0] + off[d]) / h[d];
        if (!isfinite(u)) return -5;
        const double fl = floor(u);
        if (!(fl >= 1.0 && fl <= (double)(n[d] - 2))) return -6;
        idx[d] = (int)fl;
        const double f = u - fl;
        /* w1 = f, w0 = 1 - f; d f / d p_k = x_k / h */
        w[d][0][0] = 1.0 - f;
        w[d][1][0] = f;
        for (int k = 1; k < C; ++k) {
            w[d][1][k] = x[k] / h[d];
            w[d][0][k] = -x[k] / h[d];
        }
    }
    return 0;
}

int orc2d_deposit(const orc2d_config* c, const double* state, double* n) {
    const int C = c->P + 1;
    const int64_t N = c->N;
    const int nx1 = c->nx + 1, ny1 = c->ny + 1;
    const int64_t nn = (int64_t)nx1 * ny1;
    const double hx = c->a / c->nx, hy = c->b / c->ny;
    memset(n, 0, sizeof(double) * C * nn);
    /* each macroparticle carries 1/N of the normalised density over a cell area */
    const double q = 1.0 / ((double)N * hx * hy);
    for (int64_t i = 0; i < N; ++i) {
        int idx[2];
        double w[2][2][ORC_MAXC];
        const int st = bilinear(C, state, N, i, c, idx, w);
        if (st) return st;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                dual W;
                d_mul(C, w[0][a], w[1][b], W);
                const int64_t node = (int64_t)(idx[1] + b) * nx1 + (idx[0] + a);
                for (int k = 0; k < C; ++k) n[(int64_t)k * nn + node] += q * W[k];
            }
    }
    return 0;
}

/* Eqs. for rho^lm and phi^lm: with nodes x_i = i hx (i = 0..nx, walls at 0
   and nx), rho^lm = (4 / (nx ny)) sum_ij rho_ij sin(l pi i / nx) sin(m pi j / ny)
   (the quadrature of the paper's integral on the grid), phi^lm = rho^lm /
   gamma_lm^2 with gamma_lm^2 = (l pi / a)^2 + (m pi / b)^2, and phi_ij the
   sine sums back; l, m = 1 .. n - 1. Here the Poisson equation is
   lap phi = -rho for the normalised density (eps0 and the current go into the
   kick factor 2 pi K). Separable: 1D sine sums along x, then along y. */
void orc2d_solve(const orc2d_config* c, const double* rho, double* phi) {
    const int C = c->P + 1, nx = c->nx, ny = c->ny;
    const int nx1 = nx + 1, ny1 = ny + 1;
    const int64_t nn = (int64_t)nx1 * ny1;
    double* t = (double*)malloc(sizeof(double) * nn);
    double* u = (double*)malloc(sizeof(double) * nn);
    for (int k = 0; k < C; ++k) {
        const double* r = rho + (int64_t)k * nn;
        double* p = phi + (int64_t)k * nn;
        /* forward along x: t[j][l] = sum_i r[j][i] sin(l pi i / nx) */
        for (int j = 0; j < ny1; ++j)
            for (int l = 0; l < nx1; ++l) {
                double s = 0.0;
                if (l >= 1 && l <= nx - 1)
                    for (int i = 1; i <= nx - 1; ++i) s += r[(int64_t)j * nx1 + i] * sin(PI * l * i / nx);
                t[(int64_t)j * nx1 + l] = s;
            }
        /* forward along y and the division: u[m][l] = (4/(nx ny)) sum_j t[j][l] sin(m pi j / ny) / gamma^2 */
        for (int m = 0; m < ny1; ++m)
            for (int l = 0; l < nx1; ++l) {
                double s = 0.0;
                if (m >= 1 && m <= ny - 1 && l >= 1 && l <= nx - 1) {
                    for (int j = 1; j <= ny - 1; ++j) s += t[(int64_t)j * nx1 + l] * sin(PI * m * j / ny);
                    const double al = PI * l / c->a, be = PI * m / c->b;
                    s = 4.0 / ((double)nx * ny) * s / (al * al + be * be);
                }
                u[(int64_t)m * nx1 + l] = s;
            }
        /* back along y: t[j][l] = sum_m u[m][l] sin(m pi j / ny) */
        for (int j = 0; j < ny1; ++j)
            for (int l = 0; l < nx1; ++l) {
                double s = 0.0;
                for (int m = 1; m <= ny - 1; ++m) s += u[(int64_t)m * nx1 + l] * sin(PI * m * j / ny);
                t[(int64_t)j * nx1 + l] = s;
            }
        /* back along x: p[j][i] = sum_l t[j][l] sin(l pi i / nx) */
        for (int j = 0; j < ny1; ++j)
            for (int i = 0; i < nx1; ++i) {
                double s = 0.0;
                for (int l = 1; l <= nx - 1; ++l) s += t[(int64_t)j * nx1 + l] * sin(PI * l * i / nx);
                p[(int64_t)j * nx1 + i] = s;
            }
    }
    free(t);
    free(u);
}

/* E = -grad phi by central differences at interior nodes; zero on the walls */
void orc2d_field(const orc2d_config* c, const double* phi, double* E /*[2][C][ny+1][nx+1]*/) {
    const int C = c->P + 1, nx1 = c->nx + 1, ny1 = c->ny + 1;
    const int64_t nn = (int64_t)nx1 * ny1;
    const double hx = c->a / c->nx, hy = c->b / c->ny;
    memset(E, 0, sizeof(double) * 2 * C * nn);
    for (int k = 0; k < C; ++k)
        for (int j = 1; j < ny1 - 1; ++j)
            for (int i = 1; i < nx1 - 1; ++i) {
                const double* p = phi + (int64_t)k * nn;
                const int64_t q = (int64_t)j * nx1 + i;
                E[((int64_t)0 * C + k) * nn + q] = -(p[q + 1] - p[q - 1]) / (2.0 * hx);
                E[((int64_t)1 * C + k) * nn + q] = -(p[q + nx1] - p[q - nx1]) / (2.0 * hy);
            }
}

/* M2(tau) of Sec. 4: p -= d H2 / d r tau with H2 = K phi / 2 and phi in the
   paper's normalisation (4 pi times the unit-charge potential of
   orc2d_solve): p += 2 pi K E tau, E = -grad phi (dual gather of the
   bilinear weights times the dual field) */
int orc2d_kick(const orc2d_config* c, double* state, const double* E, int64_t kick) {
    const int C = c->P + 1;
    const int64_t N = c->N;
    const int nx1 = c->nx + 1;
    const int64_t nn = (int64_t)nx1 * (c->ny + 1);
    double g0, b0, p0, brho, K;
    consts2d(c, &g0, &b0, &p0, &brho, &K);
    orc_config k3 = as3d(c);
    dual tau, two_pi_K, KI, coef;
    /* D tau of the kick's element, and the dual current (slot current_slot):
       K is linear in I, K = I (q / (2 pi eps0 p0 v0^2 gamma0^2)) */
    int e = element_of_kick(&k3, kick);
    dual_tau(&k3, e, tau);
    d_var(C, c->current_A, c->current_slot, KI);
    const double v0 = b0 * C_LIGHT;
    const double K_per_A = c->charge_e * Q_E / (2.0 * PI * EPS0 * p0 * v0 * v0 * g0 * g0);
    (void)K;
    d_cmul(C, 2.0 * PI * K_per_A, KI, two_pi_K);
    d_mul(C, two_pi_K, tau, coef);
    for (int64_t i = 0; i < N; ++i) {
        int idx[2];
        double w[2][2][ORC_MAXC];
        const int st = bilinear(C, state, N, i, c, idx, w);
        if (st) return st;
        for (int d = 0; d < 2; ++d) {
            dual Ep, W, t;
            d_const(C, 0.0, Ep);
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    d_mul(C, w[0][a], w[1][b], W);
                    const int64_t node = (int64_t)(idx[1] + b) * nx1 + (idx[0] + a);
                    dual En;
                    for (int k = 0; k < C; ++k) En[k] = E[((int64_t)d * C + k) * nn + node];
                    d_mul(C, W, En, t);
                    d_add(C, Ep, t, Ep);
                }
            double* p = state + ((int64_t)(2 * d + 1) * N + i) * C;
            d_mul(C, coef, Ep, t);
            d_add(C, p, t, p);
        }
    }
    return 0;
}

void orc2d_moments(const orc2d_config* c, const double* state, double* mom /*[2][5][C]*/) {
    orc_config k3 = as3d(c);
    k3.N = c->N;
    /* the 3D moment code over the first two planes (x, px, y, py) */
    const int C = c->P + 1;
    double* s6 = (double*)calloc((size_t)6 * c->N * C, sizeof(double));
    memcpy(s6, state, sizeof(double) * 4 * c->N * C);
    double m3[3 * 5 * ORC_MAXC];
    orc_moments(&k3, s6, m3);
    memcpy(mom, m3, sizeof(double) * 2 * 5 * C);
    free(s6);
}

int orc2d_run(const orc2d_config* c, double* state, int64_t kick0, int n_kicks, double* mom_hist) {
    const int C = c->P + 1;
    const int64_t N = c->N;
    const int64_t nn = (int64_t)(c->nx + 1) * (c->ny + 1);
    orc_config k3 = as3d(c);
    k3.N = N;
    const int kpp = kicks_per_period(&k3);
    double* rho = (double*)malloc(sizeof(double) * C * nn);
    double* phi = (double*)malloc(sizeof(double) * C * nn);
    double* E = (double*)malloc(sizeof(double) * 2 * C * nn);
    int st = 0, rec = 0;
    for (int s = 0; s < n_kicks && !st; ++s) {
        const int64_t kick = kick0 + s;
        double m[3 * 4 * ORC_MAXC];
        orc_half_map(&k3, kick, m);
        /* M1(tau/2) on the two transverse planes */
        for (int64_t i = 0; i < N; ++i)
            for (int pl = 0; pl < 2; ++pl) {
                double* u = state + ((int64_t)(2 * pl) * N + i) * C;
                double* p = state + ((int64_t)(2 * pl + 1) * N + i) * C;
                dual a, b, un, pn;
                d_mul(C, m + (pl * 4 + 0) * C, u, a); d_mul(C, m + (pl * 4 + 1) * C, p, b); d_add(C, a, b, un);
                d_mul(C, m + (pl * 4 + 2) * C, u, a); d_mul(C, m + (pl * 4 + 3) * C, p, b); d_add(C, a, b, pn);
                d_copy(C, un, u);
                d_copy(C, pn, p);
            }
        st = orc2d_deposit(c, state, rho);
        if (st) break;
        orc2d_solve(c, rho, phi);
        orc2d_field(c, phi, E);
        st = orc2d_kick(c, state, E, kick);
        if (st) break;
        for (int64_t i = 0; i < N; ++i)
            for (int pl = 0; pl < 2; ++pl) {
                double* u = state + ((int64_t)(2 * pl) * N + i) * C;
                double* p = state + ((int64_t)(2 * pl + 1) * N + i) * C;
                dual a, b, un, pn;
                d_mul(C, m + (pl * 4 + 0) * C, u, a); d_mul(C, m + (pl * 4 + 1) * C, p, b); d_add(C, a, b, un);
                d_mul(C, m + (pl * 4 + 2) * C, u, a); d_mul(C, m + (pl * 4 + 3) * C, p, b); d_add(C, a, b, pn);
                d_copy(C, un, u);
                d_copy(C, pn, p);
            }
        if (((kick + 1) % kpp == 0) || s == n_kicks - 1) {
            if (mom_hist) orc2d_moments(c, state, mom_hist + (int64_t)rec * 10 * C);
            ++rec;
        }
    }
    free(rho); free(phi); free(E);
    return st ? st : rec;
}

/* initial distribution: per plane u = sqrt(eps beta) n1, p = sqrt(eps/beta)(n2 - alpha n1), mean removed */
int orc2d_beam_init(const orc2d_config* c, const double* normals /*[4][N]*/, double* state) {
    const int C = c->P + 1;
    const int64_t N = c->N;
    double g0, b0, p0, brho, K;
    consts2d(c, &g0, &b0, &p0, &brho, &K);
    memset(state, 0, sizeof(double) * 4 * N * C);
    for (int pl = 0; pl < 2; ++pl) {
        const double eps = c->eps_n[pl] / (b0 * g0), beta = c->beta[pl], alpha = c->alpha[pl];
        double m1 = 0.0, m2 = 0.0;
        for (int64_t i = 0; i < N; ++i) { m1 += normals[(2 * pl) * N + i]; m2 += normals[(2 * pl + 1) * N + i]; }
        m1 /= (double)N;
        m2 /= (double)N;
        for (int64_t i = 0; i < N; ++i) {
            const double n1 = normals[(2 * pl) * N + i] - m1, n2 = normals[(2 * pl + 1) * N + i] - m2;
            state[((int64_t)(2 * pl) * N + i) * C] = sqrt(eps * beta) * n1;
            state[((int64_t)(2 * pl + 1) * N + i) * C] = sqrt(eps / beta) * (n2 - alpha * n1);
        }
    }
    return 0;
}
