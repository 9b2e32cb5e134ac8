/*
 * Oracle: plain FP64 CPU implementation of one time step of the double-DF
 * D2Q9 lattice Boltzmann model of Huang, Wu & Adams, "Mesoscopic lattice
 * Boltzmann modeling of the liquid-vapor phase transition" (PRL 2021).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, __graft_entry__.smoke() and
 * the CPU-baseline leg of bench.py load this file's library. It shares no
 * code, header, table or helper with the CUDA library; it is written to be
 * read against the paper, not to be fast: explicit 9x9 matrices, matrix-
 * vector products in loops, a generic Gauss-Jordan inverse of M, and push
 * streaming with explicit periodic wrap.
 *
 * State convention: f[i][y][x], g[i][y][x] hold the post-streaming
 * (pre-collision) populations at time t, i.e. the populations of which the
 * moments of Eq. 14 are taken.
 *
 * Passages followed:
 *   D2Q9 velocities ............ Supplemental Material (SM) Eq. S1
 *   transformation matrix M .... SM Eq. S2
 *   m^eq, F_m .................. SM Eq. S3a, S3b
 *   n^eq, q_m .................. SM Eq. S4a, S4b
 *   S, L and their constants ... SM Eq. S5a, S5b and the text below them
 *   Q_m, Y ..................... SM Eq. S6a, S6b; grad rho from F_pair (SM)
 *   streaming / collisions ..... Eq. 12a, 12b, 12c
 *   pair force ................. Eq. 13
 *   moments .................... Eq. 14
 *   EOS ........................ Eq. 17; p_BE = p_EOS + a rho^2 (text after
 *                                Eq. 11); p_LBE = c_s^2 (rho + eta) = p_BE
 *                                (Eq. 15 and the text after it)
 *   rho h_k = rho e_k + p_BE ... Eq. 15
 *   T from rho e_k ............. rho e_k = rho c_v T + rho |u|^2 / 2 (text
 *                                after Eq. 11)
 *
 * Not in the paper (readings of this implementation):
 *   walls: half-way bounce-back of f and g at y = -1/2 and y = ny - 1/2;
 *   fixed-temperature wall segments: anti-bounce-back of g against the
 *   rest equilibrium M^-1 n^eq(rho_w c_v T_w, T_w, u = 0) with rho_w the
 *   density of the fluid node; the ghost density for the pair force beyond
 *   a wall equals the density of the adjacent fluid node (neutral wetting);
 *   heat-conduction rate sigma_j interpolated linearly in rho between
 *   tau_j,v at rho_v and tau_j,l at rho_l (clamped), and sigma_q = sigma_j;
 *   open, heated sides for the one-dimensional Stefan problem (the bottom)
 *   and the evaporating droplet (all four sides): a ghost node beyond an
 *   open side carries the post-collision populations of its nearest fluid
 *   node with their equilibrium part moved to the open state (rho_out,
 *   T_open) at that node's velocity (non-equilibrium extrapolation);
 *   rho_out is the vapour at T_open and the liquid's saturation pressure;
 *   an optional elimination of the cubic velocity terms of the viscous
 *   stress (paragraph after Eq. 16, whose "trivial modifications" are in
 *   another paper): the equilibria of the third-order moments q_x, q_y
 *   gain 3 rho u_x u_y^2 and 3 rho u_y u_x^2 (u over c), so that the
 *   lattice's third moments Q_xyy, Q_xxy carry their rho u u u parts, and
 *   the two that D2Q9 cannot carry (Q_xxx = j_x, Q_yyy = j_y) are made up
 *   in the deviatoric normal stress: a source R_xx - R_yy in the p_xx row,
 *   R_xx = -c d_x(rho u_x^3), R_yy = -c d_y(rho u_y^3) (central differences
 *   of the neighbours' values), entering the f collision as dt (I - S/2) R
 *   like a force term. The trace (row e) is left to the model's own
 *   velocity coupling of that row in S.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, walls;
    double c, dt, G2, a, kappa, cs2;
    double R, a_t, b_t, K_EOS, cv, Cref;
    double varpi, gamma1, gamma2, beta, kS, hS, bS;
    double s0, se, seps, sj, sq, sp;
    double sig0, sige, sigeps, sigp;
    double tauj_v, tauj_l, rho_v, rho_l;
    double ax, ay;
    double T_bottom, T_top, T_hot;
    int hot_x0, hot_len;
    int open_sides;      /* open, heated sides: 1 bottom, 2 top (both need
                            walls), 4 left, 8 right (only with all four) */
    double rho_out;      /* their density (vapour at T_open and the liquid's p_s) */
    double T_open;       /* their temperature */
    int cubic;           /* eliminate the cubic velocity terms (periodic boxes) */
} orc_params;

/* SM Eq. S1: e_i / c for i = 0..8 */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* SM Eq. S2 */
static const double MM[9][9] = {
    { 1,  1,  1,  1,  1,  1,  1,  1,  1},
    {-4, -1, -1, -1, -1,  2,  2,  2,  2},
    { 4, -2, -2, -2, -2,  1,  1,  1,  1},
    { 0,  1,  0, -1,  0,  1, -1, -1,  1},
    { 0, -2,  0,  2,  0,  1, -1, -1,  1},
    { 0,  0,  1,  0, -1,  1,  1, -1, -1},
    { 0,  0, -2,  0,  2,  1,  1, -1, -1},
    { 0,  1, -1,  1, -1,  0,  0,  0,  0},
    { 0,  0,  0,  0,  0,  1, -1,  1, -1},
};

static double MI[9][9];
static int MI_ready = 0;

/* Generic Gauss-Jordan inverse with partial pivoting; M is not assumed
 * orthogonal here so that the orthogonality can be tested separately. */
static void invert_M(void)
{
    double A[9][18];
    for (int r = 0; r < 9; ++r)
        for (int k = 0; k < 18; ++k)
            A[r][k] = (k < 9) ? MM[r][k] : (k - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k < 18; ++k) { double t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
        double d = A[col][col];
        for (int k = 0; k < 18; ++k) A[col][k] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == col) continue;
            double fac = A[r][col];
            for (int k = 0; k < 18; ++k) A[r][k] -= fac * A[col][k];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int k = 0; k < 9; ++k) MI[r][k] = A[r][9 + k];
    MI_ready = 1;
}

void orc_get_M(double* out_M, double* out_Minv)
{
    if (!MI_ready) invert_M();
    for (int r = 0; r < 9; ++r)
        for (int k = 0; k < 9; ++k) { out_M[9 * r + k] = MM[r][k]; out_Minv[9 * r + k] = MI[r][k]; }
}

static void matvec(const double A[9][9], const double* v, double* out)
{
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += A[r][k] * v[k];
        out[r] = s;
    }
}

static int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* Eq. 13 weights omega(|e_i dt|^2): 1/3 on the axes, 1/12 on the diagonals */
static double pair_weight(int i) { return i == 0 ? 0.0 : (i <= 4 ? 1.0 / 3.0 : 1.0 / 12.0); }

/* Density at (x + EX, y + EY): periodic in x; periodic in y unless walls,
 * where the ghost beyond a wall carries the adjacent fluid density. */
static double rho_at(const orc_params* P, const double* rho, int x, int y)
{
    x = wrap(x, P->nx);
    if (P->walls) {
        if (y < 0) y = 0;
        if (y >= P->ny) y = P->ny - 1;
    } else {
        y = wrap(y, P->ny);
    }
    return rho[(size_t)y * P->nx + x];
}

/* Is the lattice point (x, y) beyond an open side? (x is periodic unless
 * the left and right sides are open.) */
static int beyond_open(const orc_params* P, int x, int y)
{
    return ((P->open_sides & 1) && y < 0) || ((P->open_sides & 2) && y >= P->ny) ||
           ((P->open_sides & 4) && x < 0) || ((P->open_sides & 8) && x >= P->nx);
}

/* The density the pair force sees at (x, y): beyond an open side it is
 * the fixed density rho_out, elsewhere rho_at's. */
static double rho_seen(const orc_params* P, const double* rho, int x, int y)
{
    if (beyond_open(P, x, y)) return P->rho_out;
    return rho_at(P, rho, x, y);
}

/* Eq. 17 */
static double p_eos(const orc_params* P, double rho, double T)
{
    double th = P->b_t * rho / 4.0;
    double z = (1.0 + th + th * th - th * th * th) / ((1.0 - th) * (1.0 - th) * (1.0 - th));
    return P->K_EOS * (rho * P->R * T * z - P->a_t * rho * rho);
}

static double sigma_j_of(const orc_params* P, double rho)
{
    double w = (rho - P->rho_v) / (P->rho_l - P->rho_v);
    if (w < 0.0) w = 0.0;
    if (w > 1.0) w = 1.0;
    double tau = P->tauj_v + (P->tauj_l - P->tauj_v) * w;
    return 1.0 / (tau + 0.5);
}

/* sigma_q of L (SM Eq. S5b) is not given in the paper; it is taken equal to
 * sigma_j (a linear stability analysis of the rest state rejects the
 * analogue of the S constraint, tau_j tau_q = 1/12, for tau_j >= 1/2). */
static double sigma_q_of(const orc_params* P, double rho)
{
    return sigma_j_of(P, rho);
}

/* Local macroscopic state of one node (Eq. 13, 14) */
typedef struct {
    double rho, Fpx, Fpy, Fx, Fy, ux, uy, q, rek, T;
} node_state;

static void node_macro(const orc_params* P, const double* fl, const double* gl,
                       const double* rho_f, int x, int y, node_state* s)
{
    double rho = 0.0;
    for (int i = 0; i < 9; ++i) rho += fl[i];
    /* Eq. 13 with e_i dt = (EX, EY) dx, dx = 1 */
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < 9; ++i) {
        double rn = rho_seen(P, rho_f, x + EX[i], y + EY[i]);
        sx += pair_weight(i) * rn * EX[i];
        sy += pair_weight(i) * rn * EY[i];
    }
    s->rho = rho;
    s->Fpx = P->G2 * rho * sx;
    s->Fpy = P->G2 * rho * sy;
    s->Fx = s->Fpx + rho * P->ax;
    s->Fy = s->Fpy + rho * P->ay;
    /* Eq. 14: rho u = sum e_i f_i + dt/2 F, e_i = c (EX, EY) */
    double jx = 0.0, jy = 0.0, eg = 0.0;
    for (int i = 0; i < 9; ++i) {
        jx += P->c * EX[i] * fl[i];
        jy += P->c * EY[i] * fl[i];
        eg += gl[i];
    }
    s->ux = (jx + 0.5 * P->dt * s->Fx) / rho;
    s->uy = (jy + 0.5 * P->dt * s->Fy) / rho;
    /* q = F_pair . u + rho a . u */
    s->q = s->Fx * s->ux + s->Fy * s->uy;
    s->rek = eg + 0.5 * P->dt * s->q;
    s->T = (s->rek - 0.5 * rho * (s->ux * s->ux + s->uy * s->uy)) / (rho * P->cv);
}

/* Equilibrium moments and sources of both DFs at one node (SM Eq. S3, S4),
 * with the EOS terms of Eq. 15 and Eq. 17. */
typedef struct {
    double meq[9], Fm[9], neq[9], qm[9], Qm[9];
    double S[9][9], L[9][9], Y[9][9];
} node_terms;

static void node_terms_build(const orc_params* P, const node_state* s, node_terms* t)
{
    double rho = s->rho, T = s->T;
    double uxh = s->ux / P->c, uyh = s->uy / P->c;          /* u^ = u / c */
    double Fxh = s->Fx / P->c, Fyh = s->Fy / P->c;          /* F^ = F / c */
    double u2 = uxh * uxh + uyh * uyh;
    double pBE = p_eos(P, rho, T) + P->a * rho * rho;
    double eta = pBE / P->cs2 - rho;
    double rhk = s->rek + pBE;

    double meq[9] = {rho, -2.0 * rho + 2.0 * eta + 3.0 * rho * u2, rho + P->beta * eta - 3.0 * rho * u2,
                     rho * uxh, -rho * uxh, rho * uyh, -rho * uyh,
                     rho * (uxh * uxh - uyh * uyh), rho * uxh * uyh};
    if (P->cubic) {
        /* q_x = 3 Q_xyy - 2 j_x: Q_xyy = rho u_x / 3 + rho u_x u_y^2 */
        meq[4] += 3.0 * rho * uxh * uyh * uyh;
        meq[6] += 3.0 * rho * uyh * uxh * uxh;
    }
    double FU = Fxh * uxh + Fyh * uyh;
    double Fm[9] = {0.0, 6.0 * FU, -6.0 * FU, Fxh, -Fxh, Fyh, -Fyh,
                    2.0 * Fxh * uxh - 2.0 * Fyh * uyh, Fxh * uyh + Fyh * uxh};
    double E = s->rek;
    double CT = P->Cref * T;
    double neq[9] = {E, -4.0 * E + (4.0 + P->gamma1) * CT, 4.0 * E - (4.0 - P->gamma2) * CT,
                     rhk * uxh, -rhk * uxh, rhk * uyh, -rhk * uyh, 0.0, 0.0};
    double q = s->q;
    double qm[9] = {q, P->gamma1 * q, P->gamma2 * q, q * uxh, -q * uxh, q * uyh, -q * uyh, 0.0, 0.0};
    /* grad rho from the pair force: F_pair = G^2 dx^2 rho grad rho (SM, below Eq. S6) */
    double gx = s->Fpx / (P->G2 * rho), gy = s->Fpy / (P->G2 * rho);
    double qc = P->G2 * P->dt * P->dt / 12.0;
    double g2 = gx * gx + gy * gy;
    double Qm[9] = {0.0, 6.0 * qc * g2, -6.0 * qc * g2, 0.0, 0.0, 0.0, 0.0,
                    qc * (gx * gx - gy * gy), qc * gx * gy};
    memcpy(t->meq, meq, sizeof meq);
    memcpy(t->Fm, Fm, sizeof Fm);
    memcpy(t->neq, neq, sizeof neq);
    memcpy(t->qm, qm, sizeof qm);
    memcpy(t->Qm, Qm, sizeof Qm);

    /* SM Eq. S5a */
    double we = P->se / 2.0 - 1.0, wp = P->sp / 2.0 - 1.0;
    memset(t->S, 0, sizeof t->S);
    t->S[0][0] = P->s0;
    t->S[1][1] = P->se;
    t->S[1][2] = P->kS * P->seps * we;
    t->S[1][4] = P->hS * uxh * P->sq * we;
    t->S[1][6] = P->hS * uyh * P->sq * we;
    t->S[2][2] = P->seps;
    t->S[3][3] = P->sj;
    t->S[4][4] = P->sq;
    t->S[5][5] = P->sj;
    t->S[6][6] = P->sq;
    t->S[7][4] = 2.0 * P->bS * uxh * P->sq * wp;
    t->S[7][6] = -2.0 * P->bS * uyh * P->sq * wp;
    t->S[7][7] = P->sp;
    t->S[8][4] = P->bS * uyh * P->sq * wp;
    t->S[8][6] = P->bS * uxh * P->sq * wp;
    t->S[8][8] = P->sp;

    /* SM Eq. S5b */
    double sigj = sigma_j_of(P, rho), sigq = sigma_q_of(P, rho);
    double wj = sigj / 2.0 - 1.0;
    memset(t->L, 0, sizeof t->L);
    t->L[0][0] = P->sig0;
    t->L[1][1] = P->sige;
    t->L[2][2] = P->sigeps;
    t->L[3][3] = sigj;
    t->L[3][4] = sigq * wj;
    t->L[4][4] = sigq;
    t->L[5][5] = sigj;
    t->L[5][6] = sigq * wj;
    t->L[6][6] = sigq;
    t->L[7][7] = P->sigp;
    t->L[8][8] = P->sigp;

    /* SM Eq. S6b */
    memset(t->Y, 0, sizeof t->Y);
    t->Y[3][1] = uxh / 3.0;  t->Y[3][7] = uxh;  t->Y[3][8] = 2.0 * uyh;
    t->Y[4][1] = -uxh / 3.0; t->Y[4][7] = -uxh; t->Y[4][8] = -2.0 * uyh;
    t->Y[5][1] = uyh / 3.0;  t->Y[5][7] = -uyh; t->Y[5][8] = 2.0 * uxh;
    t->Y[6][1] = -uyh / 3.0; t->Y[6][7] = uyh;  t->Y[6][8] = -2.0 * uxh;
}

/* The cubic-term source in moment space from the central differences
 * dphix = d_x(rho u_x^3), dphiy = d_y(rho u_y^3) (u over c) at the node:
 * R_xx = -c dphix, R_yy = -c dphiy, in the p_xx row as R_xx - R_yy. */
static void cubic_source(const orc_params* P, double dphix, double dphiy, double* Rm)
{
    for (int k = 0; k < 9; ++k) Rm[k] = 0.0;
    double Rxx = -P->c * dphix, Ryy = -P->c * dphiy;
    Rm[7] = Rxx - Ryy;
}

/* Collision at one node: Eq. 12b and 12c, back-transform with M^-1.
 * Rm: the cubic-term source in moment space (row p_xx), or NULL. */
static void node_collide(const orc_params* P, const double* fl, const double* gl,
                         const node_state* s, const double* Rm, double* fb, double* gb)
{
    node_terms t;
    node_terms_build(P, s, &t);
    double m[9], n[9], tmp[9], Sx[9], SQ[9], mb[9], nb[9], Lx[9], d[9], Yd[9];
    matvec(MM, fl, m);
    for (int k = 0; k < 9; ++k) tmp[k] = m[k] - t.meq[k] + 0.5 * P->dt * t.Fm[k];
    matvec(t.S, tmp, Sx);
    matvec(t.S, t.Qm, SQ);
    for (int k = 0; k < 9; ++k) mb[k] = m[k] + P->dt * t.Fm[k] - Sx[k] + SQ[k];
    if (Rm) {
        /* dt (I - S/2) R, R a source like F_m */
        double SR[9];
        matvec(t.S, Rm, SR);
        for (int k = 0; k < 9; ++k) mb[k] += P->dt * (Rm[k] - 0.5 * SR[k]);
    }

    matvec(MM, gl, n);
    for (int k = 0; k < 9; ++k) tmp[k] = n[k] - t.neq[k] + 0.5 * P->dt * t.qm[k];
    matvec(t.L, tmp, Lx);
    for (int k = 0; k < 9; ++k) d[k] = 0.5 * (m[k] + mb[k]) - t.meq[k];
    matvec(t.Y, d, Yd);
    double c2 = P->c * P->c;
    for (int k = 0; k < 9; ++k) nb[k] = n[k] + P->dt * t.qm[k] - Lx[k] + c2 * Yd[k];

    matvec(MI, mb, fb);
    matvec(MI, nb, gb);
}

/* Equilibrium populations M^-1 m^eq and M^-1 n^eq of a uniform, force-free
 * state (rho, u, T) (SM Eq. S3a, S4a). */
static void eq_populations(const orc_params* P, double rho, double ux, double uy, double T,
                           double* feq, double* geq)
{
    node_state s;
    memset(&s, 0, sizeof s);
    s.rho = rho;
    s.ux = ux;
    s.uy = uy;
    s.T = T;
    s.rek = rho * P->cv * T + 0.5 * rho * (ux * ux + uy * uy);
    node_terms t;
    node_terms_build(P, &s, &t);
    matvec(MI, t.meq, feq);
    matvec(MI, t.neq, geq);
}

/* Rest equilibrium of g against which a fixed-temperature wall reflects. */
static void g_rest_eq(const orc_params* P, double rho_w, double T_w, double* geq)
{
    double E = rho_w * P->cv * T_w, CT = P->Cref * T_w;
    double neq[9] = {E, -4.0 * E + (4.0 + P->gamma1) * CT, 4.0 * E - (4.0 - P->gamma2) * CT,
                     0, 0, 0, 0, 0, 0};
    matvec(MI, neq, geq);
}

/* Temperature of the wall reached by a link whose ghost end has abscissa xg
 * (already wrapped); <= 0 means an adiabatic wall. */
static double wall_T(const orc_params* P, int bottom, int xg)
{
    if (bottom) {
        if (P->hot_len > 0) {
            int dx = wrap(xg - P->hot_x0, P->nx);
            if (dx < P->hot_len) return P->T_hot;
        }
        return P->T_bottom;
    }
    return P->T_top;
}

static void rho_field(const orc_params* P, const double* f, double* rho)
{
    const long N = (long)P->nx * P->ny;
    #pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[i * N + p];
        rho[p] = r;
    }
}

static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* n time steps. f, g: [9][ny][nx], updated in place. */
int orc_step(const orc_params* P, double* f, double* g, int nsteps)
{
    if (!MI_ready) invert_M();
    const int nx = P->nx, ny = P->ny;
    const size_t N = (size_t)nx * ny;
    double* rho = (double*)malloc(N * sizeof(double));
    double* fn = (double*)malloc(9 * N * sizeof(double));
    double* gn = (double*)malloc(9 * N * sizeof(double));
    if (!rho || !fn || !gn) { free(rho); free(fn); free(gn); return -1; }

    double* phi = P->cubic ? (double*)malloc(2 * N * sizeof(double)) : NULL;
    if (P->cubic && !phi) { free(rho); free(fn); free(gn); return -1; }
    for (int step = 0; step < nsteps; ++step) {
        rho_field(P, f, rho);
        if (P->cubic) {
            /* rho u_x^3 and rho u_y^3 (u over c) of every node, for the
             * cubic-term source */
            #pragma omp parallel for schedule(static)
            for (long p = 0; p < (long)N; ++p) {
                double fl[9], gl[9];
                for (int i = 0; i < 9; ++i) { fl[i] = f[i * N + p]; gl[i] = g[i * N + p]; }
                node_state s;
                node_macro(P, fl, gl, rho, (int)(p % nx), (int)(p / nx), &s);
                double ux = s.ux / P->c, uy = s.uy / P->c;
                phi[p] = s.rho * ux * ux * ux;
                phi[N + p] = s.rho * uy * uy * uy;
            }
        }
        /* nodes are independent and every push target is written once */
        #pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t p = (size_t)y * nx + x;
                double fl[9], gl[9], fb[9], gb[9];
                for (int i = 0; i < 9; ++i) { fl[i] = f[i * N + p]; gl[i] = g[i * N + p]; }
                node_state s;
                node_macro(P, fl, gl, rho, x, y, &s);
                double Rm[9];
                if (P->cubic) {
                    /* periodic central differences of rho u_x^3 along x and
                     * rho u_y^3 along y */
                    double dx = 0.5 * (phi[(size_t)y * nx + wrap(x + 1, nx)] - phi[(size_t)y * nx + wrap(x - 1, nx)]);
                    double dy = 0.5 * (phi[N + (size_t)wrap(y + 1, ny) * nx + x] - phi[N + (size_t)wrap(y - 1, ny) * nx + x]);
                    cubic_source(P, dx, dy, Rm);
                }
                node_collide(P, fl, gl, &s, P->cubic ? Rm : NULL, fb, gb);
                int on_open = 0;
                for (int i = 1; i < 9; ++i) on_open |= beyond_open(P, x + EX[i], y + EY[i]);
                if (on_open) {
                    /* Open, heated sides (not in the paper, whose boundary
                     * scheme is taken from another paper): every ghost node
                     * beyond an open side whose nearest fluid node is this
                     * one carries this node's post-collision populations
                     * with their equilibrium part moved to (rho_out,
                     * T_open) at this node's velocity (non-equilibrium
                     * extrapolation), and streams into the lattice the
                     * populations that point back across the open sides.
                     * What leaves through an open side is lost. */
                    double fe[9], ge[9], fo[9], go[9];
                    eq_populations(P, s.rho, s.ux, s.uy, s.T, fe, ge);
                    eq_populations(P, P->rho_out, s.ux, s.uy, P->T_open, fo, go);
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int gx = x + dx, gy = y + dy;
                            const int ox = beyond_open(P, gx, y), oy = beyond_open(P, x, gy);
                            if (!(ox || oy) || (dx != 0 && !ox) || (dy != 0 && !oy)) continue;
                            for (int i = 1; i < 9; ++i) {
                                if ((dx != 0 && EX[i] != -dx) || (dy != 0 && EY[i] != -dy)) continue;
                                const int xd = gx + EX[i], yd = gy + EY[i];
                                if (beyond_open(P, xd, yd)) continue;
                                size_t pd = (size_t)yd * nx + wrap(xd, nx);
                                fn[i * N + pd] = fb[i] + fo[i] - fe[i];
                                gn[i * N + pd] = gb[i] + go[i] - ge[i];
                            }
                        }
                }
                /* Eq. 12a, push form */
                for (int i = 0; i < 9; ++i) {
                    int xd = x + EX[i], yd = y + EY[i];
                    if (beyond_open(P, xd, yd)) continue;
                    if (P->walls && (yd < 0 || yd >= ny)) {
                        int o = OPP[i];
                        fn[o * N + p] = fb[i];
                        double Tw = wall_T(P, yd < 0, wrap(xd, nx));
                        if (Tw > 0.0) {
                            double geq[9];
                            g_rest_eq(P, s.rho, Tw, geq);
                            gn[o * N + p] = -gb[i] + 2.0 * geq[i];
                        } else {
                            gn[o * N + p] = gb[i];
                        }
                    } else {
                        size_t pd = (size_t)wrap(yd, ny) * nx + wrap(xd, nx);
                        fn[i * N + pd] = fb[i];
                        gn[i * N + pd] = gb[i];
                    }
                }
            }
        memcpy(f, fn, 9 * N * sizeof(double));
        memcpy(g, gn, 9 * N * sizeof(double));
    }
    free(rho); free(fn); free(gn); free(phi);
    return 0;
}

/* Macroscopic fields of a state (Eq. 13, 14). Outputs [ny][nx]; also the
 * pair force and the g-moment source q so that budgets can be checked. */
int orc_moments(const orc_params* P, const double* f, const double* g,
                double* rho_o, double* ux_o, double* uy_o, double* T_o,
                double* Fpx_o, double* Fpy_o, double* q_o, double* rek_o)
{
    const int nx = P->nx, ny = P->ny;
    const size_t N = (size_t)nx * ny;
    double* rho = (double*)malloc(N * sizeof(double));
    if (!rho) return -1;
    rho_field(P, f, rho);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t p = (size_t)y * nx + x;
            double fl[9], gl[9];
            for (int i = 0; i < 9; ++i) { fl[i] = f[i * N + p]; gl[i] = g[i * N + p]; }
            node_state s;
            node_macro(P, fl, gl, rho, x, y, &s);
            if (rho_o) rho_o[p] = s.rho;
            if (ux_o) ux_o[p] = s.ux;
            if (uy_o) uy_o[p] = s.uy;
            if (T_o) T_o[p] = s.T;
            if (Fpx_o) Fpx_o[p] = s.Fpx;
            if (Fpy_o) Fpy_o[p] = s.Fpy;
            if (q_o) q_o[p] = s.q;
            if (rek_o) rek_o[p] = s.rek;
        }
    free(rho);
    return 0;
}

/* Initial populations from (rho, u, T): m = m^eq - dt/2 F_m and
 * n = n^eq - dt/2 q_m, so that Eq. 14 returns the prescribed fields. */
int orc_init(const orc_params* P, const double* rho_in, const double* ux_in,
             const double* uy_in, const double* T_in, double* f, double* g)
{
    if (!MI_ready) invert_M();
    const int nx = P->nx, ny = P->ny;
    const size_t N = (size_t)nx * ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t p = (size_t)y * nx + x;
            node_state s;
            double rho = rho_in[p];
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < 9; ++i) {
                double rn = rho_seen(P, rho_in, x + EX[i], y + EY[i]);
                sx += pair_weight(i) * rn * EX[i];
                sy += pair_weight(i) * rn * EY[i];
            }
            s.rho = rho;
            s.Fpx = P->G2 * rho * sx;
            s.Fpy = P->G2 * rho * sy;
            s.Fx = s.Fpx + rho * P->ax;
            s.Fy = s.Fpy + rho * P->ay;
            s.ux = ux_in[p];
            s.uy = uy_in[p];
            s.q = s.Fx * s.ux + s.Fy * s.uy;
            s.T = T_in[p];
            s.rek = rho * P->cv * s.T + 0.5 * rho * (s.ux * s.ux + s.uy * s.uy);
            node_terms t;
            node_terms_build(P, &s, &t);
            double m[9], n[9], fl[9], gl[9];
            for (int k = 0; k < 9; ++k) {
                m[k] = t.meq[k] - 0.5 * P->dt * t.Fm[k];
                n[k] = t.neq[k] - 0.5 * P->dt * t.qm[k];
            }
            matvec(MI, m, fl);
            matvec(MI, n, gl);
            for (int i = 0; i < 9; ++i) { f[i * N + p] = fl[i]; g[i * N + p] = gl[i]; }
        }
    return 0;
}

/* One node's collision in isolation, for unit tests of Eq. 12b/12c:
 * inputs fl, gl (9 each), rho_nb[9] = rho at x + e_i (rho_nb[0] unused),
 * dphi (may be NULL) = the central differences d_x(rho u_x^3), d_y(rho
 * u_y^3) at the node, from which the cubic-term source is formed. */
void orc_collide_node_r(const orc_params* P, const double* fl, const double* gl,
                        const double* rho_nb, const double* dphi, double* fb, double* gb, double* macro);
void orc_collide_node(const orc_params* P, const double* fl, const double* gl,
                      const double* rho_nb, double* fb, double* gb, double* macro)
{
    orc_collide_node_r(P, fl, gl, rho_nb, NULL, fb, gb, macro);
}

void orc_collide_node_r(const orc_params* P, const double* fl, const double* gl,
                        const double* rho_nb, const double* dphi, double* fb, double* gb, double* macro)
{
    if (!MI_ready) invert_M();
    node_state s;
    double rho = 0.0;
    for (int i = 0; i < 9; ++i) rho += fl[i];
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < 9; ++i) { sx += pair_weight(i) * rho_nb[i] * EX[i]; sy += pair_weight(i) * rho_nb[i] * EY[i]; }
    s.rho = rho;
    s.Fpx = P->G2 * rho * sx; s.Fpy = P->G2 * rho * sy;
    s.Fx = s.Fpx + rho * P->ax; s.Fy = s.Fpy + rho * P->ay;
    double jx = 0, jy = 0, eg = 0;
    for (int i = 0; i < 9; ++i) { jx += P->c * EX[i] * fl[i]; jy += P->c * EY[i] * fl[i]; eg += gl[i]; }
    s.ux = (jx + 0.5 * P->dt * s.Fx) / rho;
    s.uy = (jy + 0.5 * P->dt * s.Fy) / rho;
    s.q = s.Fx * s.ux + s.Fy * s.uy;
    s.rek = eg + 0.5 * P->dt * s.q;
    s.T = (s.rek - 0.5 * rho * (s.ux * s.ux + s.uy * s.uy)) / (rho * P->cv);
    double Rm[9];
    if (dphi) cubic_source(P, dphi[0], dphi[1], Rm);
    node_collide(P, fl, gl, &s, dphi ? Rm : NULL, fb, gb);
    if (macro) {
        macro[0] = s.rho; macro[1] = s.ux; macro[2] = s.uy; macro[3] = s.T;
        macro[4] = s.Fx; macro[5] = s.Fy; macro[6] = s.q; macro[7] = s.rek;
    }
}
