/*
 * Plain FP64 CPU oracle for the dual-number 3D space-charge PIC step.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library,
 * its Python binding) may include, link or call this code. Only the tests,
 * __graft_entry__.smoke() and the cpu_baseline leg of bench.py use it.
 *
 * The oracle is written for readability against the paper, not for speed:
 * a runtime-sized dual number (value plus P first derivatives, Sec. 2,
 * Eqs. 1-4), the split-operator step M1(tau/2) M2(tau) M1(tau/2) (Sec. 4,
 * Eq. "map"), the thick-quadrupole maps (Eq. "quadtr" and its defocusing
 * twin, written in dual variables as in the equation following "Dk, Dtau"),
 * cloud-in-cell deposition and gathering (Sec. 4, linear deposition), an
 * open-boundary Hockney convolution with an integrated Green's function,
 * central finite-difference fields, and the dual emittance of Sec. 4
 * (Eqs. for D<x^2>, D<px^2>, D<x px>).
 *
 * Where the paper is silent (3D, rest frame, Green's function, grid geometry,
 * longitudinal map) the oracle takes one written reading; every such reading
 * is listed with the repository's design notes.
 *
 * Layouts (all row-major, all FP64):
 *   particle state  [6][N][C]   coordinates (x, px, y, py, z, delta)
 *   grid channel    [C][nz][ny][nx]
 *   field           [3][C][nz][ny][nx]   (Ex, Ey, Ez), rest-frame V/m
 *   moments         [3][5][C]   planes (x,y,z) x (<u>,<p>,<u^2>,<u p>,<p^2>)
 *   geometry        [6]         origin x,y,z (m, lab), spacing hx,hy,hz (lab)
 *
 * Return codes: 0 ok, -1 invalid argument, -5 non-finite value,
 * -6 particle outside the grid.
 */
#ifndef ADPIC_ORACLE_H
#define ADPIC_ORACLE_H
#include <stdint.h>

#define ORC_MAXC 32

/* one element of a beamline: type 0 drift, 1 thick quadrupole of normalised
   strength k (1/m^2; > 0 focuses in x, defocuses in y); slot_L, slot_k are
   the derivative slots of L and k (-1 = constant) */
typedef struct {
    int32_t type, slot_L, slot_k, pad;
    double L, k;
} orc_element;

typedef struct {
    int32_t P;            /* derivative slots; C = P + 1 channels */
    int32_t nx, ny, nz;   /* grid nodes per dimension (powers of two, >= 8) */
    int64_t N;            /* macroparticles */
    double kinetic_eV;    /* reference kinetic energy (eV) */
    double mass_eV;       /* rest energy (eV) */
    double charge_e;      /* particle charge in units of e */
    double bunch_charge_C;/* physical bunch charge (C) */
    double eps_n[3];      /* normalized rms emittance per plane (m rad) */
    double alpha[3];      /* Twiss alpha per plane at the start */
    double beta[3];       /* Twiss beta per plane at the start (m) */
    int32_t twiss_slot[6];/* slots of (alpha_x, beta_x, eps_x, alpha_y, beta_y, eps_y); -1 = constant */
    double L[5];          /* element lengths D1, QF, D2, QD, D3 (m) */
    double g[2];          /* gradients of QF, QD (T/m) */
    int32_t kicks[5];     /* space-charge kicks per element */
    int32_t lat_slot[7];  /* slots of (L_D1, L_QF, g_QF, L_D2, L_QD, g_QD, L_D3); -1 = constant */
    /* a general beamline in place of the FODO period (n_line > 0): its
       elements in beam order and the space-charge kicks of each; the period
       (moment records, kick schedule) is then the whole beamline */
    int32_t n_line, pad_line;
    const orc_element* line;
    const int32_t* line_kicks;
    /* slot of the bunch charge as an AD variable (Sec. 4: beam current as a
       dual input), -1 = constant: the macroparticle charge Q / N is then a
       dual number */
    int32_t charge_slot;
    /* slot of the kinetic energy as an AD variable (Sec. 4: beam parameters
       as dual inputs), -1 = constant: gamma0, beta0 gamma0, B rho and the kick
       constants are then dual, and so are the rest-frame z spacing gamma0 hz
       of the Green's function and of the field */
    int32_t energy_slot;
} orc_config;

/* derived constants: gamma0, beta0, p0 (kg m/s), Brho (T m), kappa_perp, kappa_z, q_macro (C), q (C) */
void orc_constants(const orc_config* cfg, double out[8]);
/* the same as duals (energy_slot): out[6][C] = gamma0, beta0 gamma0, Brho, kappa_perp, kappa_z, 1/gamma0^2 */
void orc_dual_constants(const orc_config* cfg, double* out);

/* dual arithmetic, exposed for the pins: op 0 add, 1 sub, 2 mul, 3 div,
   4 sqrt, 5 sin, 6 cos, 7 sinh, 8 cosh, 9 exp (g ignored for unary ops) */
void orc_dual_op(int op, int C, const double* f, const double* g, double* out);
/* the five-variable test function of Sec. 3, with all five seeded: out[6] */
void orc_testfn(const double x[5], double out[6]);

/* FFT of one complex sequence of power-of-two length n (sign -1 forward,
   +1 inverse, unnormalised), in place on split re/im arrays */
int orc_fft1d(double* re, double* im, int n, int sign);

/* cell-averaged 1/(4 pi eps0 r) over the box of size (hx,hy,hz) centred at (x,y,z) */
double orc_igf(double x, double y, double z, double hx, double hy, double hz);
/* the same at the node offset (x, y, kz hz) and its derivative with respect to
   hz (the centre moves with hz): out[2] = (G, dG/dhz) */
void orc_igf_dhz(double x, double y, double kz, double hx, double hy, double hz, double out[2]);

int orc_beam_init(const orc_config* cfg, const double* normals /*[6][N]*/, double* state);
void orc_half_map(const orc_config* cfg, int64_t kick, double* m /*[3][4][C]*/);
void orc_apply_half_map(const orc_config* cfg, double* state, int64_t kick);
int orc_geometry(const orc_config* cfg, const double* state, double* geom);
int orc_deposit(const orc_config* cfg, const double* state, const double* geom, double* rho);
void orc_green(const orc_config* cfg, const double* geom, double* G /*[2nz][2ny][2nx]*/);
/* dG/dE (E the kinetic energy, eV) on the same doubled grid, through the
   rest-frame spacing gamma0 hz */
void orc_green_denergy(const orc_config* cfg, const double* geom, double* GE);
int orc_solve(const orc_config* cfg, const double* geom, const double* rho, double* phi);
int orc_solve_direct(const orc_config* cfg, const double* geom, const double* rho, double* phi);
void orc_field(const orc_config* cfg, const double* geom, const double* phi, double* E);
int orc_gather(const orc_config* cfg, const double* state, const double* geom, const double* E,
               double* Ep /*[3][N][C]*/);
int orc_kick(const orc_config* cfg, double* state, const double* geom, const double* E, int64_t kick);
void orc_moments(const orc_config* cfg, const double* state, double* mom);
void orc_emittance(const orc_config* cfg, const double* mom, double* eps /*[3][C]*/);

/* Run n_kicks split steps starting at global kick index kick0.
   geom_mode 0: geometry from the particles; 1: same and record into
   geom_io[n_kicks][6]; 2: replay geom_io (frozen geometry).
   Moments are recorded into mom_hist[r][3][5][C] at every period end and
   after the last kick; the return value is the number of records (>= 0)
   or a negative status. */
int orc_run(const orc_config* cfg, double* state, int64_t kick0, int n_kicks,
            double* mom_hist, double* geom_io, int geom_mode);

/* ---- single-particle dual optics (Sec. 3) ---- */

/* dual 2x2 matrices of the beamline (elements in beam order):
   m[plane x, y][m11, m12, m21, m22][C] */
void orc_beamline_matrix(int P, const orc_element* el, int n, double* m);
/* Twiss transport (Sec. 3, Eq. 5) through the beamline from constant
   twiss0[4] = (beta_x, alpha_x, beta_y, alpha_y): out[4][C] */
void orc_twiss(int P, const orc_element* el, int n, const double* twiss0, double* out);
/* periodic Twiss functions of a cell, out[4][C]; -1 if the cell is unstable */
int orc_periodic_twiss(int P, const orc_element* el, int n, double* out);
/* particles x0[N][4] (x, px, y, py) through the beamline n_repeat times,
   element by element: out[N][4][C] */
void orc_track(int P, const orc_element* el, int n, int64_t n_repeat, int64_t N, const double* x0, double* out);

/* ---- 2D PIC in a rectangular conducting pipe (Sec. 4) ---- */

typedef struct {
    int32_t P;            /* derivative slots; C = P + 1 */
    int32_t nx, ny;       /* cells per dimension: nodes 0..nx, 0..ny, walls at 0 and n */
    int32_t current_slot; /* slot of the beam current as an AD variable, -1 = constant */
    int64_t N;            /* macroparticles */
    double a, b;          /* pipe widths (m); the beam axis is the pipe centre */
    double kinetic_eV, mass_eV, charge_e, current_A;
    double eps_n[2], alpha[2], beta[2];   /* per plane x, y (constant Twiss) */
    double L[5], g[2];
    int32_t kicks[5];
    int32_t lat_slot[7];
} orc2d_config;

/* gamma0, beta0, p0 (kg m/s), B rho (T m), K = q I / (2 pi eps0 p0 v0^2 gamma0^2) */
void orc2d_constants(const orc2d_config* c, double out[5]);
int orc2d_beam_init(const orc2d_config* c, const double* normals /*[4][N]*/, double* state /*[4][N][C]*/);
/* normalised density (integral 1 over the pipe) on the nodes: n[C][ny+1][nx+1] */
int orc2d_deposit(const orc2d_config* c, const double* state, double* n);
/* lap phi = -n with phi = 0 on the walls by the sine series of Sec. 4 */
void orc2d_solve(const orc2d_config* c, const double* n, double* phi);
void orc2d_field(const orc2d_config* c, const double* phi, double* E /*[2][C][ny+1][nx+1]*/);
int orc2d_kick(const orc2d_config* c, double* state, const double* E, int64_t kick);
void orc2d_moments(const orc2d_config* c, const double* state, double* mom /*[2][5][C]*/);
/* split steps; records [r][2][5][C] at every period end and after the last kick */
int orc2d_run(const orc2d_config* c, double* state, int64_t kick0, int n_kicks, double* mom_hist);

#endif
