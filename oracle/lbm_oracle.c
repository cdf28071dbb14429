/*
 * lbm_oracle.c -- plain FP64 reference of the D3Q19 BGK collide-and-stream
 * update (test infrastructure only).
 *
 * This file is the oracle that the CUDA path is checked against.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it;
 * the product library never links, calls or includes it, and it shares no
 * table, header or helper with the CUDA sources.
 *
 * What it computes.  Fu & Song (arXiv 2208.05429) merge two collision-
 * streaming cycles of a D3Q19 lattice (Sec. 3, Alg. 1; Sec. 4.1, Alg. 2;
 * Sec. 4.2, Alg. 3) and state that the merged solvers reproduce the plain
 * single-step solver exactly (Sec. 5.1, verification of the four solvers on
 * the same cavity).  The paper never writes down the lattice, the collision
 * or the boundary rule; they are the Palabos defaults it builds on.  The
 * oracle therefore is the plain definition of one time step, written out in
 * the textbook form the method reaches:
 *
 *   lattice    D3Q19, c_0 = 0, six face vectors (w = 1/18), twelve edge
 *              vectors (w = 1/36), w_0 = 1/3, c_s^2 = 1/3.  Directions 1..9
 *              are the vectors whose first non-zero component (x, y, z order)
 *              is -1 -- the half of the neighbours the swap streams to
 *              (Sec. 3) -- and direction i+9 is the opposite of i.  The
 *              same rule orders D3Q15 (w_0 = 2/9, faces 1/9, corners 1/72)
 *              and D3Q27 (w_0 = 8/27, faces 2/27, edges 1/54, corners
 *              1/216), the other cubic sets the paper's dependency guard
 *              covers (Sec. 4.1); cfg.q selects one, c_s^2 = 1/3 on all
 *              three, and every formula below holds on each of them except
 *              the MRT basis, which is D3Q19's.
 *   collision  BGK with Guo forcing, omega = 1/tau:
 *                rho = sum f_i,  u = (sum f_i c_i + F/2) / rho
 *                feq_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
 *                S_i   = w_i (3 (c_i - u) + 9 (c_i.u) c_i) . F
 *                f*_i  = f_i - omega (f_i - feq_i) + (1 - omega/2) S_i
 *              or, as one of the "collision models" the paper's solver
 *              builds on (Sec. 1), the two-relaxation-time (TRT) form: with
 *              the symmetric and antisymmetric parts a^+-_i = (a_i +- a_opp(i))/2
 *              of f, feq and S, the rates omega+ = 1/tau and omega- given by
 *              the "magic" product Lambda = (1/omega+ - 1/2)(1/omega- - 1/2),
 *                f*_i  = f_i - omega+ (f+_i - feq+_i) - omega- (f-_i - feq-_i)
 *                        + (1 - omega+/2) S+_i + (1 - omega-/2) S-_i
 *              (omega- = omega+ gives back BGK), or the regularised BGK form:
 *              f - feq replaced by its projection on the Hermite
 *              polynomials up to second order before relaxing,
 *                f*_i  = feq_i + (1 - omega) w_i (3 c_i . J + (9/2) Q_i : Pi)
 *                        + (1 - omega/2) S_i
 *              with J = sum_i (f_i - feq_i) c_i, Pi = sum_i (f_i - feq_i) c_i c_i
 *              and Q_i = c_i c_i - I/3; or a multiple-relaxation-time form
 *              that relaxes the Hermite moments of f - feq of order three
 *              and four with rates s3 and s4 (orc_collide_cell_mrt).
 *   streaming  f_i(x + c_i, t+1) = f*_i(x); periodic axes wrap; a link that
 *              leaves the box across a non-periodic face is a wall link
 *              (half-way bounce-back):
 *                f_opp(i)(x, t+1) = f*_i(x) - 6 w_i rho_w (c_i . u_w)
 *              with u_w the lid velocity when one of the faces crossed is a
 *              LID face (the lid takes precedence at edges and corners),
 *              zero otherwise.
 *
 * The state at step n is the post-stream population f^n in the canonical
 * layout f[i][z][y][x] (x fastest).  Everything is double precision and is
 * evaluated in the order written above, cell by cell, with no blocking or
 * fusion beyond the one-cell collide-then-scatter of the definition.
 *
 * The adjoint (orc_adjoint_step, orc_adjoint_seed) is the hand-derived
 * discrete adjoint of the step above, with rho_w constant so that the lid
 * term has no derivative.  It has no counterpart in the paper.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_LID = 2 };
enum { FORCE_NONE = 0, FORCE_UNIFORM = 1, FORCE_FIELD = 2 };
enum { COLL_BGK = 0, COLL_TRT = 1, COLL_REG = 2, COLL_MRT = 3 };

/* The velocity sets, each in the half-neighbour order described above:
 * direction 0 is the rest vector, directions 1 .. H (H = (q - 1) / 2) are the
 * vectors whose first non-zero component is -1, and direction i + H is the
 * opposite of i.  D3Q19 is the paper's lattice; D3Q15 (six faces, eight
 * corners) and D3Q27 (six faces, twelve edges, eight corners) are the other
 * two cubic sets for which the paper's dependency guard holds (Sec. 4.1). */
#define QMAX 27

typedef struct {
    int q;
    int c[QMAX][3];
    double w[QMAX];
} orc_lat;

static const orc_lat D3Q19 = {
    19,
    {
        {0, 0, 0},
        {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {-1, -1, 0}, {-1, 1, 0},
        {-1, 0, -1}, {-1, 0, 1}, {0, -1, -1}, {0, -1, 1},
        {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
        {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1},
    },
    {
        1.0 / 3.0,
        1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0,
        1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
        1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0,
        1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    },
};

/* D3Q15: w_0 = 2/9, faces 1/9, corners 1/72. */
static const orc_lat D3Q15 = {
    15,
    {
        {0, 0, 0},
        {-1, 0, 0}, {0, -1, 0}, {0, 0, -1},
        {-1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}, {-1, 1, 1},
        {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
        {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1},
    },
    {
        2.0 / 9.0,
        1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
        1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
        1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
        1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
    },
};

/* D3Q27: w_0 = 8/27, faces 2/27, edges 1/54, corners 1/216. */
static const orc_lat D3Q27 = {
    27,
    {
        {0, 0, 0},
        {-1, 0, 0}, {0, -1, 0}, {0, 0, -1},
        {-1, -1, 0}, {-1, 1, 0}, {-1, 0, -1}, {-1, 0, 1}, {0, -1, -1}, {0, -1, 1},
        {-1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}, {-1, 1, 1},
        {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
        {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1},
        {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1},
    },
    {
        8.0 / 27.0,
        2.0 / 27.0, 2.0 / 27.0, 2.0 / 27.0,
        1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0,
        1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0,
        2.0 / 27.0, 2.0 / 27.0, 2.0 / 27.0,
        1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0, 1.0 / 54.0,
        1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0, 1.0 / 216.0,
    },
};

/* The lattice of a configuration's q (0 or 19: D3Q19). */
static const orc_lat *lat_of(int32_t q) { return q == 15 ? &D3Q15 : q == 27 ? &D3Q27 : &D3Q19; }

static int opp_of(const orc_lat *L, int i)
{
    const int h = L->q / 2;
    return i == 0 ? 0 : (i <= h ? i + h : i - h);
}

typedef struct {
    int64_t nx, ny, nz;
    double tau;
    int32_t bc[6];          /* x-, x+, y-, y+, z-, z+ */
    double u_lid[3];
    double rho_wall;
    int32_t force_mode;
    double force_uniform[3];
    const double *force_field; /* [3][N] canonical, used when FORCE_FIELD */
    int32_t collision;         /* COLL_BGK, COLL_TRT, COLL_REG or COLL_MRT */
    double trt_lambda;         /* Lambda of the TRT form */
    double mrt_s3, mrt_s4;     /* MRT: rates of the third- and fourth-order moments */
    int32_t q;                 /* lattice: 15, 19 or 27 velocities (0: 19) */
} orc_cfg;

static int64_t ncells(const orc_cfg *g) { return g->nx * g->ny * g->nz; }

static int64_t cell_index(const orc_cfg *g, int64_t x, int64_t y, int64_t z)
{
    return (z * g->ny + y) * g->nx + x;
}

/* Body force acting on one cell. */
static void cell_force(const orc_cfg *g, int64_t cell, double F[3])
{
    const int64_t n = ncells(g);
    for (int a = 0; a < 3; ++a) {
        if (g->force_mode == FORCE_UNIFORM)
            F[a] = g->force_uniform[a];
        else if (g->force_mode == FORCE_FIELD)
            F[a] = g->force_field[a * n + cell];
        else
            F[a] = 0.0;
    }
}

/* Follow the link from cell (x,y,z) along c_i.  Returns 1 and the target
 * cell when the link stays inside the (periodically wrapped) box, 0 for a
 * wall link; *lid tells whether a LID face is among the faces crossed. */
static int link_target(const orc_cfg *g, int64_t x, int64_t y, int64_t z, int i,
                       int64_t *target, int *lid)
{
    const int *c = lat_of(g->q)->c[i];
    int64_t p[3] = {x + c[0], y + c[1], z + c[2]};
    const int64_t n[3] = {g->nx, g->ny, g->nz};
    int wall = 0;
    *lid = 0;
    for (int a = 0; a < 3; ++a) {
        if (p[a] < 0 || p[a] >= n[a]) {
            const int face = 2 * a + (p[a] < 0 ? 0 : 1);
            if (g->bc[face] == BC_PERIODIC) {
                p[a] = (p[a] + n[a]) % n[a];
            } else {
                wall = 1;
                if (g->bc[face] == BC_LID) *lid = 1;
            }
        }
    }
    if (wall) return 0;
    *target = cell_index(g, p[0], p[1], p[2]);
    return 1;
}

/* Moving-wall correction 6 w_i rho_w (c_i . u_w) of a wall link. */
static double wall_term(const orc_cfg *g, int i, int lid)
{
    if (!lid) return 0.0;
    const orc_lat *L = lat_of(g->q);
    const double cu = L->c[i][0] * g->u_lid[0] + L->c[i][1] * g->u_lid[1] + L->c[i][2] * g->u_lid[2];
    return 6.0 * L->w[i] * g->rho_wall * cu;
}

/* ------------------------------------------------------------------ */
/* lattice tables, equilibrium, collision                              */
/* ------------------------------------------------------------------ */

/* The tables of lattice q (15, 19 or 27; 0 means 19): c[q][3], w[q], opp[q]. */
void orc_lattice_q(int32_t q, int32_t *c, double *w, int32_t *opp)
{
    const orc_lat *L = lat_of(q);
    for (int i = 0; i < L->q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L->c[i][a];
        w[i] = L->w[i];
        opp[i] = opp_of(L, i);
    }
}

void orc_lattice(int32_t *c /* [19][3] */, double *w /* [19] */, int32_t *opp /* [19] */)
{
    orc_lattice_q(19, c, w, opp);
}

static void equilibrium_l(const orc_lat *L, double rho, const double *u, double *feq)
{
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->q; ++i) {
        const double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        feq[i] = L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

void orc_equilibrium_q(int32_t q, double rho, const double *u, double *feq) { equilibrium_l(lat_of(q), rho, u, feq); }

void orc_equilibrium(double rho, const double *u, double *feq) { equilibrium_l(&D3Q19, rho, u, feq); }

/* rho, u = (sum f_i c_i + F/2) / rho, and per direction feq_i and the Guo
 * term S_i of one cell (the ingredients every collision below shares). */
static void collide_terms(const orc_lat *L, const double *f, const double *F, double *rho_out, double u[3],
                          double *feq, double *S)
{
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) m[a] += f[i] * L->c[i][a];
    }
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / rho;
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    for (int i = 0; i < L->q; ++i) {
        const double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        const double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
        feq[i] = L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
        S[i] = L->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
    }
    *rho_out = rho;
}

/* BGK collision of one cell. */
static void collide_bgk(const orc_lat *L, double tau, const double *f, const double *F, double *fstar)
{
    double rho, u[3], feq[QMAX], S[QMAX];
    collide_terms(L, f, F, &rho, u, feq, S);
    const double omega = 1.0 / tau;
    for (int i = 0; i < L->q; ++i) fstar[i] = f[i] - omega * (f[i] - feq[i]) + (1.0 - 0.5 * omega) * S[i];
}

/* TRT collision of one cell: the BGK ingredients above, relaxed by parts. */
static void collide_trt(const orc_lat *L, double tau, double lambda, const double *f, const double *F, double *fstar)
{
    double rho, u[3], feq[QMAX], S[QMAX];
    collide_terms(L, f, F, &rho, u, feq, S);
    const double omega_p = 1.0 / tau;
    const double omega_m = 1.0 / (0.5 + lambda / (tau - 0.5));
    for (int i = 0; i < L->q; ++i) {
        const int o = opp_of(L, i);
        const double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
        const double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
        const double sp = 0.5 * (S[i] + S[o]), sm = 0.5 * (S[i] - S[o]);
        fstar[i] = f[i] - omega_p * (fp - ep) - omega_m * (fm - em) + (1.0 - 0.5 * omega_p) * sp +
                   (1.0 - 0.5 * omega_m) * sm;
    }
}

/* Regularised BGK collision of one cell: the non-equilibrium part f - feq is
 * replaced by its projection on the Hermite polynomials up to second order,
 * which keeps its momentum (-F/2 with a body force, zero without) and its
 * stress and drops every higher ("ghost") moment, and then relaxed:
 *   J_a   = sum_i (f_i - feq_i) c_ia,   Pi_ab = sum_i (f_i - feq_i) c_ia c_ib
 *   f1_i  = w_i (3 c_ia J_a + (9/2) (c_ia c_ib - delta_ab / 3) Pi_ab)
 *   f*_i  = feq_i + (1 - omega) f1_i + (1 - omega/2) S_i
 * with feq, S and u as in the BGK collision above. */
static void collide_reg(const orc_lat *L, double tau, const double *f, const double *F, double *fstar)
{
    double rho, u[3], feq[QMAX], S[QMAX], J[3] = {0.0, 0.0, 0.0}, Pi[3][3] = {{0.0}};
    collide_terms(L, f, F, &rho, u, feq, S);
    const double omega = 1.0 / tau;
    for (int i = 0; i < L->q; ++i)
        for (int a = 0; a < 3; ++a) {
            J[a] += (f[i] - feq[i]) * L->c[i][a];
            for (int b = 0; b < 3; ++b) Pi[a][b] += (f[i] - feq[i]) * L->c[i][a] * L->c[i][b];
        }
    for (int i = 0; i < L->q; ++i) {
        double q = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) q += (L->c[i][a] * L->c[i][b] - (a == b ? 1.0 / 3.0 : 0.0)) * Pi[a][b];
        const double cJ = L->c[i][0] * J[0] + L->c[i][1] * J[1] + L->c[i][2] * J[2];
        const double f1 = L->w[i] * (3.0 * cJ + 4.5 * q);
        fstar[i] = feq[i] + (1.0 - omega) * f1 + (1.0 - 0.5 * omega) * S[i];
    }
}

void orc_collide_cell(double tau, const double *f, const double *F, double *fstar)
{
    collide_bgk(&D3Q19, tau, f, F, fstar);
}

void orc_collide_cell_trt(double tau, double lambda, const double *f, const double *F, double *fstar)
{
    collide_trt(&D3Q19, tau, lambda, f, F, fstar);
}

void orc_collide_cell_reg(double tau, const double *f, const double *F, double *fstar)
{
    collide_reg(&D3Q19, tau, f, F, fstar);
}

/* One cell of lattice q with collision BGK, TRT (lambda) or regularised BGK. */
void orc_collide_cell_q(int32_t q, int32_t collision, double tau, double lambda, const double *f, const double *F,
                        double *fstar)
{
    const orc_lat *L = lat_of(q);
    if (collision == COLL_TRT) collide_trt(L, tau, lambda, f, F, fstar);
    else if (collision == COLL_REG) collide_reg(L, tau, f, F, fstar);
    else collide_bgk(L, tau, f, F, fstar);
}

#define Q19 19

/* Multiple-relaxation-time collision of one cell in Hermite moments.  The
 * 19 functions of c
 *   1;  x, y, z;  xx-1/3, yy-1/3, zz-1/3, xy, xz, yz;
 *   xxy-y/3, xxz-z/3, xyy-x/3, yyz-z/3, xzz-x/3, yzz-y/3;
 *   (xx-1/3)(yy-1/3), (xx-1/3)(zz-1/3), (yy-1/3)(zz-1/3)
 * are made orthogonal in sum_i w_i a(c_i) b(c_i) by Gram-Schmidt in this
 * order (on D3Q19 the fourth-order ones are not orthogonal to the second-order
 * ones, nor the third-order ones to each other), giving H_p with norms N_p and
 * orders 0 .. 4.  The non-equilibrium part n = f - feq is expanded as
 * n_i = w_i sum_p (sum_j H_p(c_j) n_j) H_p(c_i) / N_p, the part of order k is
 * relaxed with rate s_k (omega = 1/tau up to second order, s3, s4 above it):
 *   f*_i = feq_i + sum_p (1 - s_order(p)) w_i b_p H_p(c_i) / N_p + (1 - omega/2) S_i.
 * s3 = s4 = omega gives BGK, s3 = s4 = 1 the regularised form, and (without a
 * force) s3 = omega-, s4 = omega the TRT form. */
static double mrt_H[Q19][Q19], mrt_N[Q19];  /* basis H_p(c_i) and norms */
static int mrt_order[Q19];
static int mrt_ready;

static void mrt_basis(void)
{
    if (mrt_ready) return;
    for (int i = 0; i < Q19; ++i) {
        const double x = D3Q19.c[i][0], y = D3Q19.c[i][1], z = D3Q19.c[i][2], t = 1.0 / 3.0;
        const double v[Q19] = {1.0, x, y, z, x * x - t, y * y - t, z * z - t, x * y, x * z, y * z,
                             x * x * y - y * t, x * x * z - z * t, x * y * y - x * t, y * y * z - z * t,
                             x * z * z - x * t, y * z * z - y * t, (x * x - t) * (y * y - t),
                             (x * x - t) * (z * z - t), (y * y - t) * (z * z - t)};
        for (int p = 0; p < Q19; ++p) mrt_H[p][i] = v[p];
    }
    static const int order[Q19] = {0, 1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 4, 4, 4};
    for (int p = 0; p < Q19; ++p) {
        mrt_order[p] = order[p];
        for (int q = 0; q < p; ++q) {
            double d = 0.0;
            for (int i = 0; i < Q19; ++i) d += D3Q19.w[i] * mrt_H[p][i] * mrt_H[q][i];
            for (int i = 0; i < Q19; ++i) mrt_H[p][i] -= d / mrt_N[q] * mrt_H[q][i];
        }
        double nn = 0.0;
        for (int i = 0; i < Q19; ++i) nn += D3Q19.w[i] * mrt_H[p][i] * mrt_H[p][i];
        mrt_N[p] = nn;
    }
    mrt_ready = 1;
}

void orc_collide_cell_mrt(double tau, double s3, double s4, const double *f, const double *F, double *fstar)
{
    mrt_basis();
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q19; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) m[a] += f[i] * D3Q19.c[i][a];
    }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / rho;
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const double omega = 1.0 / tau;
    double feq[Q19], S[Q19], n[Q19], b[Q19];
    for (int i = 0; i < Q19; ++i) {
        const double cu = D3Q19.c[i][0] * u[0] + D3Q19.c[i][1] * u[1] + D3Q19.c[i][2] * u[2];
        const double cF = D3Q19.c[i][0] * F[0] + D3Q19.c[i][1] * F[1] + D3Q19.c[i][2] * F[2];
        feq[i] = D3Q19.w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
        S[i] = D3Q19.w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
        n[i] = f[i] - feq[i];
    }
    for (int p = 0; p < Q19; ++p) {
        b[p] = 0.0;
        for (int i = 0; i < Q19; ++i) b[p] += mrt_H[p][i] * n[i];
    }
    for (int i = 0; i < Q19; ++i) {
        double r = 0.0;
        for (int p = 0; p < Q19; ++p) {
            const double sp = mrt_order[p] <= 2 ? omega : (mrt_order[p] == 3 ? s3 : s4);
            r += (1.0 - sp) * D3Q19.w[i] * b[p] * mrt_H[p][i] / mrt_N[p];
        }
        fstar[i] = feq[i] + r + (1.0 - 0.5 * omega) * S[i];
    }
}

/* The collision the configuration selects. */
static void collide_cfg(const orc_cfg *g, const double *f, const double *F, double *fstar)
{
    const orc_lat *L = lat_of(g->q);
    if (g->collision == COLL_TRT) collide_trt(L, g->tau, g->trt_lambda, f, F, fstar);
    else if (g->collision == COLL_REG) collide_reg(L, g->tau, f, F, fstar);
    else if (g->collision == COLL_MRT) orc_collide_cell_mrt(g->tau, g->mrt_s3, g->mrt_s4, f, F, fstar);
    else collide_bgk(L, g->tau, f, F, fstar);
}

/* ------------------------------------------------------------------ */
/* field operations                                                    */
/* ------------------------------------------------------------------ */

/* f = feq(rho, u) in every cell; rho == NULL means 1, u == NULL means 0. */
void orc_init_equilibrium(const orc_cfg *g, const double *rho, const double *u, double *f)
{
    const orc_lat *L = lat_of(g->q);
    const int64_t n = ncells(g);
    for (int64_t cell = 0; cell < n; ++cell) {
        const double r = rho ? rho[cell] : 1.0;
        double uc[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int a = 0; a < 3; ++a) uc[a] = u[a * n + cell];
        double feq[QMAX];
        equilibrium_l(L, r, uc, feq);
        for (int i = 0; i < L->q; ++i) f[i * n + cell] = feq[i];
    }
}

/* One time step, f_in -> f_out (two lattices, f_out fully overwritten). */
void orc_step(const orc_cfg *g, const double *f_in, double *f_out)
{
    const orc_lat *L = lat_of(g->q);
    if (g->collision == COLL_MRT) mrt_basis();  /* once, before the threads read it */
    const int64_t n = ncells(g);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < g->nz; ++z)
        for (int64_t y = 0; y < g->ny; ++y)
            for (int64_t x = 0; x < g->nx; ++x) {
                const int64_t cell = cell_index(g, x, y, z);
                double f[QMAX], fs[QMAX], F[3];
                for (int i = 0; i < L->q; ++i) f[i] = f_in[i * n + cell];
                cell_force(g, cell, F);
                collide_cfg(g, f, F, fs);
                for (int i = 0; i < L->q; ++i) {
                    int64_t t;
                    int lid;
                    if (link_target(g, x, y, z, i, &t, &lid))
                        f_out[i * n + t] = fs[i];
                    else
                        f_out[opp_of(L, i) * n + cell] = fs[i] - wall_term(g, i, lid);
                }
            }
}

/* f^{t+1} at selected cells only: out[k][19] for the cells xyz[k] = (x,y,z).
 * Each population is fetched from the cell it streams out of (the cell
 * x - c_i, or x itself across a wall link), which is collided on the way --
 * the same rule as orc_step read from the receiving side, so that single
 * cells of a large lattice can be checked without stepping all of it. */
void orc_step_cells(const orc_cfg *g, const double *f_in, const int64_t *xyz, int64_t count, double *out)
{
    const orc_lat *L = lat_of(g->q);
    if (g->collision == COLL_MRT) mrt_basis();
    const int64_t n = ncells(g);
    for (int64_t k = 0; k < count; ++k) {
        const int64_t x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
        for (int i = 0; i < L->q; ++i) {
            int64_t src;
            int lid;
            double f[QMAX], fs[QMAX], F[3];
            if (link_target(g, x, y, z, opp_of(L, i), &src, &lid)) {
                for (int j = 0; j < L->q; ++j) f[j] = f_in[j * n + src];
                cell_force(g, src, F);
                collide_cfg(g, f, F, fs);
                out[k * L->q + i] = fs[i];
            } else {
                const int64_t self = cell_index(g, x, y, z);
                for (int j = 0; j < L->q; ++j) f[j] = f_in[j * n + self];
                cell_force(g, self, F);
                collide_cfg(g, f, F, fs);
                out[k * L->q + i] = fs[opp_of(L, i)] - wall_term(g, opp_of(L, i), lid);
            }
        }
    }
}

/* Threads of the OpenMP loops from now on (n >= 1; n <= 0 leaves them),
 * returning the number in effect.  Only the host timing of the oracle sets
 * it; the results do not depend on it (every cell is computed the same way). */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* nsteps time steps in place on f; tmp is a second lattice of the same size. */
void orc_run(const orc_cfg *g, double *f, int64_t nsteps, double *tmp)
{
    const orc_lat *L = lat_of(g->q);
    const int64_t n = ncells(g);
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_step(g, f, tmp);
        memcpy(f, tmp, sizeof(double) * (size_t)(L->q * n));
    }
}

/* rho[N] and u[3][N] of the post-stream state, u including half the force. */
void orc_moments(const orc_cfg *g, const double *f, double *rho, double *u)
{
    const orc_lat *L = lat_of(g->q);
    const int64_t n = ncells(g);
    for (int64_t cell = 0; cell < n; ++cell) {
        double r = 0.0, m[3] = {0.0, 0.0, 0.0}, F[3];
        for (int i = 0; i < L->q; ++i) {
            r += f[i * n + cell];
            for (int a = 0; a < 3; ++a) m[a] += f[i * n + cell] * L->c[i][a];
        }
        cell_force(g, cell, F);
        rho[cell] = r;
        for (int a = 0; a < 3; ++a) u[a * n + cell] = (m[a] + 0.5 * F[a]) / r;
    }
}

/* out = {sum rho, sum_x sum_i f_i c_ix, ...y, ...z, sum 1/2 rho |u|^2},
 * summed cell by cell in canonical order. */
void orc_reduce(const orc_cfg *g, const double *f, double *out)
{
    const orc_lat *L = lat_of(g->q);
    const int64_t n = ncells(g);
    double M = 0.0, P[3] = {0.0, 0.0, 0.0}, KE = 0.0;
    for (int64_t cell = 0; cell < n; ++cell) {
        double r = 0.0, m[3] = {0.0, 0.0, 0.0}, F[3];
        for (int i = 0; i < L->q; ++i) {
            r += f[i * n + cell];
            for (int a = 0; a < 3; ++a) m[a] += f[i * n + cell] * L->c[i][a];
        }
        cell_force(g, cell, F);
        double usq = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double ua = (m[a] + 0.5 * F[a]) / r;
            usq += ua * ua;
        }
        M += r;
        for (int a = 0; a < 3; ++a) P[a] += m[a];
        KE += 0.5 * r * usq;
    }
    out[0] = M;
    out[1] = P[0];
    out[2] = P[1];
    out[3] = P[2];
    out[4] = KE;
}

/* ------------------------------------------------------------------ */
/* discrete adjoint (no counterpart in the paper)                      */
/* ------------------------------------------------------------------ */

/* Reverse of orc_step: given f_t (the state the forward step started from)
 * and lam_next = dL/df^{t+1}, write lam_t = dL/df^t and add dL/dF (per cell,
 * through this step) to gF[3][N]. */
void orc_adjoint_step(const orc_cfg *g, const double *f_t, const double *lam_next,
                      double *lam_t, double *gF)
{
    const orc_lat *L = lat_of(g->q);
    const int64_t n = ncells(g);
    const double omega = 1.0 / g->tau;
    const double k = 1.0 - 0.5 * omega;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < g->nz; ++z)
        for (int64_t y = 0; y < g->ny; ++y)
            for (int64_t x = 0; x < g->nx; ++x) {
                const int64_t cell = cell_index(g, x, y, z);
                double f[QMAX], F[3], mu[QMAX];
                for (int i = 0; i < L->q; ++i) f[i] = f_t[i * n + cell];
                cell_force(g, cell, F);
                double rho = 0.0, m[3] = {0.0, 0.0, 0.0}, u[3];
                for (int i = 0; i < L->q; ++i) {
                    rho += f[i];
                    for (int a = 0; a < 3; ++a) m[a] += f[i] * L->c[i][a];
                }
                for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / rho;
                const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                /* mu_i = dL/df*_i: transpose of the streaming map */
                for (int i = 0; i < L->q; ++i) {
                    int64_t t;
                    int lid;
                    if (link_target(g, x, y, z, i, &t, &lid))
                        mu[i] = lam_next[i * n + t];
                    else
                        mu[i] = lam_next[opp_of(L, i) * n + cell];
                }
                double A = 0.0, B[3] = {0.0, 0.0, 0.0}, S[3] = {0.0, 0.0, 0.0};
                double G[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < L->q; ++i) {
                    const double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
                    const double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
                    /* d feq_i / d rho */
                    A += mu[i] * L->w[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                    for (int a = 0; a < 3; ++a) {
                        /* d feq_i / d u_a */
                        B[a] += mu[i] * L->w[i] * rho * (3.0 * L->c[i][a] + 9.0 * cu * L->c[i][a] - 3.0 * u[a]);
                        /* d S_i / d u_a */
                        S[a] += mu[i] * L->w[i] * (-3.0 * F[a] + 9.0 * cF * L->c[i][a]);
                        /* d S_i / d F_a at fixed u */
                        G[a] += mu[i] * L->w[i] * (3.0 * (L->c[i][a] - u[a]) + 9.0 * cu * L->c[i][a]);
                    }
                }
                double E[3];
                for (int a = 0; a < 3; ++a) E[a] = omega * B[a] + k * S[a];
                for (int j = 0; j < L->q; ++j) {
                    double v = (1.0 - omega) * mu[j] + omega * A;
                    for (int a = 0; a < 3; ++a) v += E[a] * (L->c[j][a] - u[a]) / rho;
                    lam_t[j * n + cell] = v;
                }
                for (int a = 0; a < 3; ++a) gF[a * n + cell] += k * G[a] + E[a] / (2.0 * rho);
            }
}

/* Seed of the reverse sweep for a loss of the output moments (rho, u) of
 * state f: lam = dL/df, gF += dL/dF through u's half-force term.
 * dLdrho may be NULL (loss independent of rho). */
void orc_adjoint_seed(const orc_cfg *g, const double *f, const double *dLdrho,
                      const double *dLdu, double *lam, double *gF)
{
    const orc_lat *L = lat_of(g->q);
    const int64_t n = ncells(g);
    for (int64_t cell = 0; cell < n; ++cell) {
        double r = 0.0, m[3] = {0.0, 0.0, 0.0}, F[3], u[3];
        for (int i = 0; i < L->q; ++i) {
            r += f[i * n + cell];
            for (int a = 0; a < 3; ++a) m[a] += f[i * n + cell] * L->c[i][a];
        }
        cell_force(g, cell, F);
        for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / r;
        for (int j = 0; j < L->q; ++j) {
            double v = dLdrho ? dLdrho[cell] : 0.0;
            for (int a = 0; a < 3; ++a) v += dLdu[a * n + cell] * (L->c[j][a] - u[a]) / r;
            lam[j * n + cell] = v;
        }
        for (int a = 0; a < 3; ++a) gF[a * n + cell] += dLdu[a * n + cell] / (2.0 * r);
    }
}
