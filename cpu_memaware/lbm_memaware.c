/*
 * lbm_memaware.c -- the paper's own CPU algorithms for the D3Q19 update, as
 * a host comparator timed beside the GPU path (Fu & Song, arXiv 2208.05429):
 *
 *   mem_fuse              the fused swap LBM of Sec. 3, Alg. 1: one time step
 *                         per sweep, single copy, swap streaming;
 *   mem_two_step_prism    the sequential memory-aware LBM of Sec. 4.1,
 *                         Alg. 2: two time steps per sweep, prism traversal
 *                         with stride `tile`;
 *   mem_two_step_prism_omp  its OpenMP form of Sec. 4.2, Alg. 3: X-slabs per
 *                         thread, the intersection layers handled in three
 *                         stages with three barriers per two time steps.
 *
 * Lattice, collision and walls are the ones the GPU path computes: D3Q19,
 * BGK with (optional, uniform) Guo forcing, half-way bounce-back on every
 * face, the moving-lid term -6 w_i rho_w (c_i . u_w) on a link that crosses
 * a lid face (the lid takes precedence at edges and corners).  All six faces
 * are walls or lids (the paper's cavity); the swap traversal cannot wrap a
 * periodic axis within one sweep, so periodic faces are rejected.  Double
 * precision throughout, like the paper's solvers.
 *
 * Coordinates.  The paper's (X, Y, Z) are the lattice's (z, y, x): X is the
 * layer axis (slowest, split among threads, the lid on the top layer of the
 * cavity), Z the row axis (fastest).  The populations are stored cell by
 * cell (array of structures, as in the paper's Palabos-based solvers):
 * f[((z * ny + y) * nx + x) * 19 + i].
 *
 * The swap scheme (Sec. 3).  Directions 1..9 point to the neighbours that
 * come earlier in memory (first non-zero of (c_z, c_y, c_x) is -1), i + 9 is
 * the opposite of i.  A cell collides and reverts (stores f*_i in slot
 * opp(i)); its swap_stream then exchanges, for i = 1..9, its slot i + 9 with
 * slot i of the neighbour x + c_i.  After both cells of a link have collided
 * and reverted, that one exchange leaves both post-stream values in place,
 * so a link may be streamed at any time between the two collisions at its
 * ends and the step after.  A link that leaves the box is not exchanged: the
 * reverted value already sits in the bounce-back slot (plus the lid term).
 *
 * The dependency checker.  Built with -DMEM_CHECK, every collision and every
 * link exchange checks, with counters per cell and per link, that it happens
 * exactly when the scheme allows (a collision only after all 18 incoming
 * links of the previous step are streamed; a link only after both its cells
 * have collided this step, and once), and counts violations.  The tests run
 * every traversal through it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define H 9 /* directions 1..H are exchanged with a neighbour; i + H is opposite */

enum { MEM_WALL = 1, MEM_LID = 2 };
enum { MEM_OK = 0, MEM_EINVAL = -1, MEM_ENOMEM = -2 };

/* c_i as (c_x, c_y, c_z).  1..9: the first non-zero of (c_z, c_y, c_x) is -1
 * (the earlier neighbours in memory); 10..18: their opposites, same order. */
static const int CV[Q][3] = {
    {0, 0, 0},
    {0, 0, -1}, {-1, 0, -1}, {1, 0, -1}, {0, -1, -1}, {0, 1, -1},
    {0, -1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 0, 0},
    {0, 0, 1}, {1, 0, 1}, {-1, 0, 1}, {0, 1, 1}, {0, -1, 1},
    {0, 1, 0}, {1, 1, 0}, {-1, 1, 0}, {1, 0, 0},
};

typedef struct {
    int64_t nx, ny, nz;
    double tau;
    int32_t bc[6];       /* x-, x+, y-, y+, z-, z+: MEM_WALL or MEM_LID */
    double u_lid[3];
    double rho_wall;
    int32_t force_mode;  /* 0: none, 1: uniform */
    double force_uniform[3];
} mem_cfg;

/* Per-run constants. */
typedef struct {
    int64_t lx, ly, lz;  /* the paper's extents: lx = nz, ly = ny, lz = nx */
    int64_t off[Q];      /* memory offset (cells) of the neighbour x + c_i */
    double w[Q];
    double L[Q];         /* lid term of a link bounced into slot k */
    double omega, kf, F[3];
    int force;
    int lid[6];
} mem_run;

static double weight(int i)
{
    const int n = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
    return n == 0 ? 1.0 / 3.0 : (n == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

static int setup(const mem_cfg *g, mem_run *r)
{
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->tau > 0.5)) return MEM_EINVAL;
    for (int k = 0; k < 6; ++k)
        if (g->bc[k] != MEM_WALL && g->bc[k] != MEM_LID) return MEM_EINVAL;
    if (g->force_mode != 0 && g->force_mode != 1) return MEM_EINVAL;
    r->lx = g->nz;
    r->ly = g->ny;
    r->lz = g->nx;
    for (int i = 0; i < Q; ++i) {
        r->off[i] = ((int64_t)CV[i][2] * g->ny + CV[i][1]) * g->nx + CV[i][0];
        r->w[i] = weight(i);
        const double cu = CV[i][0] * g->u_lid[0] + CV[i][1] * g->u_lid[1] + CV[i][2] * g->u_lid[2];
        r->L[i] = 6.0 * r->w[i] * g->rho_wall * cu;
    }
    r->omega = 1.0 / g->tau;
    r->kf = 1.0 - 0.5 * r->omega;
    r->force = g->force_mode == 1;
    for (int a = 0; a < 3; ++a) r->F[a] = r->force ? g->force_uniform[a] : 0.0;
    for (int k = 0; k < 6; ++k) r->lid[k] = g->bc[k] == MEM_LID;
    return MEM_OK;
}

/* ------------------------------------------------------------ checker */
#ifdef MEM_CHECK
static int64_t *chk_coll;   /* collisions done, per cell */
static int64_t *chk_back;   /* exchanges of link (x, x + c_i), i = 1..9, per cell */
static int64_t *chk_fwall;  /* bounce-backs of the wall link (x, x - c_i), per cell */
static int64_t chk_violations;

static void chk_bad(void) { __atomic_fetch_add(&chk_violations, 1, __ATOMIC_RELAXED); }
static int64_t chk_get(const int64_t *a, int64_t k) { return __atomic_load_n(&a[k], __ATOMIC_ACQUIRE); }
static void chk_set(int64_t *a, int64_t k, int64_t v) { __atomic_store_n(&a[k], v, __ATOMIC_RELEASE); }
#endif

/* ------------------------------------------------------------ cell operations */
static int64_t cell_of(const mem_run *r, int64_t X, int64_t Y, int64_t Z) { return (X * r->ly + Y) * r->lz + Z; }

static int on_box(const mem_run *r, int64_t X, int64_t Y, int64_t Z)
{
    return X == 0 || X == r->lx - 1 || Y == 0 || Y == r->ly - 1 || Z == 0 || Z == r->lz - 1;
}

/* Does the link from (X, Y, Z) along c_i leave the box, and across a lid? */
static int leaves(const mem_run *r, int64_t X, int64_t Y, int64_t Z, int i, int *lid)
{
    const int64_t tz = Z + CV[i][0], ty = Y + CV[i][1], tx = X + CV[i][2];
    int out = 0;
    *lid = 0;
    if (tz < 0 || tz >= r->lz) { out = 1; *lid |= r->lid[tz < 0 ? 0 : 1]; }
    if (ty < 0 || ty >= r->ly) { out = 1; *lid |= r->lid[ty < 0 ? 2 : 3]; }
    if (tx < 0 || tx >= r->lx) { out = 1; *lid |= r->lid[tx < 0 ? 4 : 5]; }
    return out;
}

/* Collide the cell at p and revert: slot opp(i) receives f*_i (BGK with Guo
 * forcing, omega = 1/tau, u = (sum f_i c_i + F/2) / rho). */
static void collide_revert(const mem_run *r, double *f, int64_t p, int64_t X, int64_t Y, int64_t Z)
{
#ifdef MEM_CHECK
    const int64_t k = chk_get(chk_coll, p) + 1;
    for (int i = 1; i <= H; ++i) {
        if (chk_get(chk_back, p * H + i - 1) != k - 1) chk_bad();
        int lid;
        if (leaves(r, X, Y, Z, i + H, &lid)) {
            if (chk_get(chk_fwall, p * H + i - 1) != k - 1) chk_bad();
        } else if (chk_get(chk_back, (p - r->off[i]) * H + i - 1) != k - 1) {
            chk_bad();
        }
    }
    chk_set(chk_coll, p, k);
#else
    (void)X; (void)Y; (void)Z;
#endif
    double *c = f + p * Q;
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
#pragma GCC unroll 19
    for (int i = 0; i < Q; ++i) {
        rho += c[i];
        m[0] += c[i] * CV[i][0];
        m[1] += c[i] * CV[i][1];
        m[2] += c[i] * CV[i][2];
    }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * r->F[a]) / rho;
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double uF = u[0] * r->F[0] + u[1] * r->F[1] + u[2] * r->F[2];
    double fs[Q];
#pragma GCC unroll 19
    for (int i = 0; i < Q; ++i) {
        const double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        const double feq = r->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
        double v = c[i] - r->omega * (c[i] - feq);
        if (r->force) {
            const double cF = CV[i][0] * r->F[0] + CV[i][1] * r->F[1] + CV[i][2] * r->F[2];
            v += r->kf * (r->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF));
        }
        fs[i] = v;
    }
    c[0] = fs[0];
    for (int i = 1; i <= H; ++i) {
        c[i + H] = fs[i];
        c[i] = fs[i + H];
    }
}

/* swap_stream of an inner cell (all 18 neighbours exist): exchange slot
 * i + 9 of p with slot i of p + c_i, i = 1..9. */
static void swap_bulk(const mem_run *r, double *f, int64_t p)
{
    double *c = f + p * Q;
#pragma GCC unroll 9
    for (int i = 1; i <= H; ++i) {
        double *n = f + (p + r->off[i]) * Q;
#ifdef MEM_CHECK
        const int64_t k = chk_get(chk_coll, p);
        if (chk_get(chk_coll, p + r->off[i]) != k || chk_get(chk_back, p * H + i - 1) != k - 1) chk_bad();
        chk_set(chk_back, p * H + i - 1, k);
#endif
        const double t = c[i + H];
        c[i + H] = n[i];
        n[i] = t;
    }
}

/* boundary_swap_stream of a cell on the bounding box: the exchanges whose
 * neighbour exists; a link that leaves the box keeps the reverted value in
 * the bounce-back slot, plus the lid term when it crosses a lid face (both
 * for the nine links to earlier neighbours and for the nine to later ones,
 * whose slots nobody else writes). */
static void swap_boundary(const mem_run *r, double *f, int64_t p, int64_t X, int64_t Y, int64_t Z)
{
    double *c = f + p * Q;
    for (int i = 1; i <= H; ++i) {
        int lid;
#ifdef MEM_CHECK
        const int64_t k = chk_get(chk_coll, p);
#endif
        if (leaves(r, X, Y, Z, i, &lid)) {
            if (lid) c[i + H] += r->L[i + H];
#ifdef MEM_CHECK
            if (chk_get(chk_back, p * H + i - 1) != k - 1) chk_bad();
            chk_set(chk_back, p * H + i - 1, k);
#endif
        } else {
            double *n = f + (p + r->off[i]) * Q;
#ifdef MEM_CHECK
            if (chk_get(chk_coll, p + r->off[i]) != k || chk_get(chk_back, p * H + i - 1) != k - 1) chk_bad();
            chk_set(chk_back, p * H + i - 1, k);
#endif
            const double t = c[i + H];
            c[i + H] = n[i];
            n[i] = t;
        }
        if (leaves(r, X, Y, Z, i + H, &lid)) {
            if (lid) c[i] += r->L[i];
#ifdef MEM_CHECK
            if (chk_get(chk_fwall, p * H + i - 1) != k - 1) chk_bad();
            chk_set(chk_fwall, p * H + i - 1, k);
#endif
        }
    }
}

/* The paper's helpers (Alg. 2): boundary_cell_comp, adaptive_collide_stream
 * and the stream half of the latter. */
static void cell_comp(const mem_run *r, double *f, int64_t X, int64_t Y, int64_t Z)
{
    const int64_t p = cell_of(r, X, Y, Z);
    collide_revert(r, f, p, X, Y, Z);
    if (on_box(r, X, Y, Z)) swap_boundary(r, f, p, X, Y, Z);
    else swap_bulk(r, f, p);
}

static void stream_only(const mem_run *r, double *f, int64_t X, int64_t Y, int64_t Z)
{
    const int64_t p = cell_of(r, X, Y, Z);
    if (on_box(r, X, Y, Z)) swap_boundary(r, f, p, X, Y, Z);
    else swap_bulk(r, f, p);
}

static void collide_only(const mem_run *r, double *f, int64_t X, int64_t Y, int64_t Z)
{
    collide_revert(r, f, cell_of(r, X, Y, Z), X, Y, Z);
}

/* ------------------------------------------------------------ traversals */
static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

/* What a traversal does at each visited cell. */
typedef struct walk walk;
typedef void (*visit_fn)(const walk *, int64_t X, int64_t Y, int64_t Z);
struct walk {
    const mem_run *r;
    double *f;
    int64_t S, E;  /* the layers [S, E] traversed (the whole box, or one thread's slab) */
    visit_fn visit;
};

/* Prism traversal of the layers [S, E] with stride `tile` (Sec. 4.1, Fig. 4):
 * prisms of tile x tile x tile cells whose rows shift one cell back in Y
 * per layer and one cell back in Z per row and per layer, following the
 * swap dependencies, so that when a cell has done its first step the cell
 * one back in X, Y and Z has all it needs for its second.  Within a prism
 * the walk goes along Z, then Y, then up in X; prisms follow one another in
 * Z, then Y, then X.  Truncated at the box faces. */
static void prism_walk(const walk *w, int64_t tile)
{
    const int64_t ly = w->r->ly, lz = w->r->lz;
    for (int64_t oX = w->S; oX <= w->E; oX += tile)
        for (int64_t oY = 0; oY <= ly + tile - 2; oY += tile)
            for (int64_t oZ = 0; oZ <= lz + 2 * (tile - 1) - 1; oZ += tile) {
                int64_t dx = 0;
                for (int64_t X = oX; X <= imin(oX + tile - 1, w->E); ++X, ++dx) {
                    const int64_t minY = oY - dx, maxY = minY + tile - 1;
                    int64_t dy = 0;
                    for (int64_t Y = imax(minY, 0); Y <= imin(maxY, ly - 1); ++Y, ++dy) {
                        const int64_t minZ = oZ - dx - dy, maxZ = minZ + tile - 1;
                        for (int64_t Z = imax(minZ, 0); Z <= imin(maxZ, lz - 1); ++Z) w->visit(w, X, Y, Z);
                    }
                }
            }
}

/* boundary_neighbor_handler (Alg. 2): the second step of the cells of layer
 * X-1 that the (-1, -1, -1) rule never reaches -- the last column (Z = lz-1),
 * the last row (Y = ly-1) and their corner -- once their inputs are
 * complete.  `op` is the second-step operation (collide and stream, or
 * collide and revert only).
 *
 * The last row.  As printed, the handler completes (X-1, ly-1, Z-1) when
 * (X, ly-1, Z) is visited.  That cell's second-step exchange along
 * (dX, dY, dZ) = (0, -1, +1), one of D3Q19's swap directions, meets
 * (X-1, ly-2, Z), whose second collision the (-1, -1, -1) rule makes only
 * at the next visit, (X, ly-1, Z+1): the exchange would move that cell's
 * inputs instead of its outputs.  So the last-row cell completed here is
 * the one two back in Z, (X-1, ly-1, Z-2), whose latest input, the second
 * step of (X-1, ly-2, Z-1), the (-1, -1, -1) rule has just made; the last
 * two cells of the row follow the last column at the row's end. */
typedef void (*cell_op)(const mem_run *, double *, int64_t, int64_t, int64_t);
static void neighbor_handler(const mem_run *r, double *f, int64_t X, int64_t Y, int64_t Z, cell_op op)
{
    if (X == 0) return;
    const int zl = Z == r->lz - 1, yl = Y == r->ly - 1;
    if (yl && Z >= 2) op(r, f, X - 1, Y, Z - 2);
    if (zl && Y > 0) op(r, f, X - 1, Y - 1, Z);
    if (yl && zl) {
        if (Z >= 1) op(r, f, X - 1, Y, Z - 1);
        op(r, f, X - 1, Y, Z);
    }
}

/* One plane's cells in memory order, one operation each. */
static void layer_op(const mem_run *r, double *f, int64_t X, cell_op op)
{
    for (int64_t Y = 0; Y < r->ly; ++Y)
        for (int64_t Z = 0; Z < r->lz; ++Z) op(r, f, X, Y, Z);
}

/* The cells of the bounding box in memory order: collide and revert
 * (collide = 1) or boundary_swap_stream (collide = 0). */
static void box_pass(const mem_run *r, double *f, int collide)
{
    const int64_t lx = r->lx, ly = r->ly, lz = r->lz;
    for (int64_t X = 0; X < lx; ++X)
        for (int64_t Y = 0; Y < ly; ++Y) {
            const int row = X == 0 || X == lx - 1 || Y == 0 || Y == ly - 1;
            for (int64_t Z = 0; Z < lz; Z += (row || lz < 2) ? 1 : lz - 1) {
                const int64_t p = cell_of(r, X, Y, Z);
                if (collide) collide_revert(r, f, p, X, Y, Z);
                else swap_boundary(r, f, p, X, Y, Z);
            }
        }
}

/* Stage II of Alg. 1: collide and swap_stream on the inner cells in memory
 * order (their earlier neighbours are inner cells already done or box cells
 * collided in Stage I). */
static void bulk_pass(const mem_run *r, double *f)
{
    for (int64_t X = 1; X < r->lx - 1; ++X)
        for (int64_t Y = 1; Y < r->ly - 1; ++Y)
            for (int64_t Z = 1; Z < r->lz - 1; ++Z) {
                const int64_t p = cell_of(r, X, Y, Z);
                collide_revert(r, f, p, X, Y, Z);
                swap_bulk(r, f, p);
            }
}

/* Alg. 1, one time step: collide and revert on the bounding box (Stage I),
 * the inner cells (Stage II), boundary_swap_stream on the box (Stage III). */
static void fuse_step(const mem_run *r, double *f)
{
    box_pass(r, f, 1);
    bulk_pass(r, f);
    box_pass(r, f, 0);
}

/* Alg. 2, the visit of cell (X, Y, Z): its first step, the second step of
 * the cell one back in X, Y and Z, and the boundary neighbours. */
static void visit_seq(const walk *w, int64_t X, int64_t Y, int64_t Z)
{
    cell_comp(w->r, w->f, X, Y, Z);
    if (X > 0 && Y > 0 && Z > 0) cell_comp(w->r, w->f, X - 1, Y - 1, Z - 1);
    neighbor_handler(w->r, w->f, X, Y, Z, cell_comp);
}

/* Alg. 2, two time steps: the prism walk over the whole box, then the
 * second step of the top layer (which no visit reaches). */
static void two_step_seq(const mem_run *r, double *f, int64_t tile)
{
    walk w = {r, f, 0, r->lx - 1, visit_seq};
    prism_walk(&w, tile);
    layer_op(r, f, r->lx - 1, cell_comp);
}

/* Alg. 3, Stage II: the visit of cell (X, Y, Z) in the slab [S, E]. */
static void visit_omp(const walk *w, int64_t X, int64_t Y, int64_t Z)
{
    const mem_run *r = w->r;
    double *f = w->f;
    if (X != w->E && (X == 0 || Y == 0 || Z == 0)) {
        /* case 0: the first row and column of a layer, and the first layer
         * of the box: first step only (no cell one back exists) */
        cell_comp(r, f, X, Y, Z);
    } else if (X == w->S) {
        /* case 1: the slab's first layer, first step (the layer below, the
         * other thread's intersection, was collided in Stage I) */
        cell_comp(r, f, X, Y, Z);
    } else if (X == w->S + 1) {
        /* case 2: first step; the second collision of the cells of layer S
         * it completes, without their stream (their links to the layer
         * below wait for its second collision, Stage III) */
        cell_comp(r, f, X, Y, Z);
        collide_only(r, f, X - 1, Y - 1, Z - 1);
        neighbor_handler(r, f, X, Y, Z, collide_only);
    } else if (X == w->E) {
        /* case 3: the intersection layer, collided in Stage I: its first
         * stream, then the second step of the layer below */
        stream_only(r, f, X, Y, Z);
        if (Y > 0 && Z > 0) cell_comp(r, f, X - 1, Y - 1, Z - 1);
        neighbor_handler(r, f, X, Y, Z, cell_comp);
    } else {
        /* case 4: the other layers, as in Alg. 2 */
        cell_comp(r, f, X, Y, Z);
        cell_comp(r, f, X - 1, Y - 1, Z - 1);
        neighbor_handler(r, f, X, Y, Z, cell_comp);
    }
}

/* Alg. 3, two time steps with `nslab` X-slabs of at least three layers (the
 * first lx % nslab slabs one layer taller), one per thread; threads beyond
 * nslab only join the barriers. */
static void two_step_omp(const mem_run *r, double *f, int64_t tile, int nthreads)
{
#pragma omp parallel num_threads(nthreads)
    {
        int nt = 1, tid = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        tid = omp_get_thread_num();
#endif
        const int64_t nslab = imax(1, imin(nt, r->lx / 3));
        const int64_t base = r->lx / nslab, rem = r->lx % nslab;
        const int active = tid < nslab;
        const int64_t S = tid * base + imin(tid, rem);
        const int64_t E = S + base + (tid < rem ? 1 : 0) - 1;
        /* Stage I: first collide and revert on the intersection layer */
        if (active) layer_op(r, f, E, collide_only);
#pragma omp barrier
        /* Stage II: the slab's prism walk, cases 0-4 */
        if (active) {
            walk w = {r, f, S, E, visit_omp};
            prism_walk(&w, tile);
        }
#pragma omp barrier
        /* Stage III: second collide and stream on the intersection layer,
         * then the second stream of the slab's first layer */
        if (active) layer_op(r, f, E, cell_comp);
#pragma omp barrier
        if (active) layer_op(r, f, S, stream_only);
    }
}

/* ------------------------------------------------------------ checker set-up */
#ifdef MEM_CHECK
static int chk_begin(const mem_run *r)
{
    const int64_t n = r->lx * r->ly * r->lz;
    chk_coll = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    chk_back = (int64_t *)calloc((size_t)n * H, sizeof(int64_t));
    chk_fwall = (int64_t *)calloc((size_t)n * H, sizeof(int64_t));
    if (!chk_coll || !chk_back || !chk_fwall) {
        free(chk_coll); free(chk_back); free(chk_fwall);
        chk_coll = chk_back = chk_fwall = NULL;
        return MEM_ENOMEM;
    }
    return MEM_OK;
}

/* After `steps` time steps every cell has collided `steps` times and every
 * link (and every bounce-back) has been streamed `steps` times. */
static void chk_end(const mem_run *r, int64_t steps)
{
    for (int64_t X = 0; X < r->lx; ++X)
        for (int64_t Y = 0; Y < r->ly; ++Y)
            for (int64_t Z = 0; Z < r->lz; ++Z) {
                const int64_t p = cell_of(r, X, Y, Z);
                if (chk_coll[p] != steps) chk_bad();
                for (int i = 1; i <= H; ++i) {
                    int lid;
                    if (chk_back[p * H + i - 1] != steps) chk_bad();
                    if (leaves(r, X, Y, Z, i + H, &lid) && chk_fwall[p * H + i - 1] != steps) chk_bad();
                }
            }
    free(chk_coll); free(chk_back); free(chk_fwall);
    chk_coll = chk_back = chk_fwall = NULL;
}
#endif

/* ------------------------------------------------------------ C entry points */

/* Directions in this library's order: c[3 i + a] (a = x, y, z), w[i].  Either
 * may be NULL. */
int mem_lattice(int32_t *c, double *w)
{
    for (int i = 0; i < Q; ++i) {
        if (c) for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        if (w) w[i] = weight(i);
    }
    return MEM_OK;
}

/* 1 in the build with the dependency checker, else 0. */
int mem_checked(void)
{
#ifdef MEM_CHECK
    return 1;
#else
    return 0;
#endif
}

/* Violations the checker has counted since the last call to
 * mem_check_reset (-1 without the checker). */
int64_t mem_check_violations(void)
{
#ifdef MEM_CHECK
    return __atomic_load_n(&chk_violations, __ATOMIC_RELAXED);
#else
    return -1;
#endif
}

void mem_check_reset(void)
{
#ifdef MEM_CHECK
    __atomic_store_n(&chk_violations, 0, __ATOMIC_RELAXED);
#endif
}

/* nsteps time steps of Alg. 1 on f (the cell-by-cell layout above, this
 * library's direction order; post-stream populations in and out). */
int mem_fuse(const mem_cfg *g, double *f, int64_t nsteps)
{
    mem_run r;
    const int rc = setup(g, &r);
    if (rc != MEM_OK) return rc;
    if (!f || nsteps < 0) return MEM_EINVAL;
#ifdef MEM_CHECK
    if (chk_begin(&r) != MEM_OK) return MEM_ENOMEM;
#endif
    for (int64_t s = 0; s < nsteps; ++s) fuse_step(&r, f);
#ifdef MEM_CHECK
    chk_end(&r, nsteps);
#endif
    return MEM_OK;
}

/* nsteps time steps with Alg. 2: nsteps / 2 two-step sweeps with prism
 * stride `tile` (>= 1; 0 = one prism over the whole box, i.e. plain memory
 * order, the paper's "2-step LBM" without prisms) and, for an odd nsteps, a
 * last step of Alg. 1. */
int mem_two_step_prism(const mem_cfg *g, double *f, int64_t nsteps, int64_t tile)
{
    mem_run r;
    const int rc = setup(g, &r);
    if (rc != MEM_OK) return rc;
    if (!f || nsteps < 0 || tile < 0) return MEM_EINVAL;
    if (tile == 0) tile = r.lx + r.ly + r.lz;
#ifdef MEM_CHECK
    if (chk_begin(&r) != MEM_OK) return MEM_ENOMEM;
#endif
    for (int64_t s = 0; s + 1 < nsteps; s += 2) two_step_seq(&r, f, tile);
    if (nsteps % 2) fuse_step(&r, f);
#ifdef MEM_CHECK
    chk_end(&r, nsteps);
#endif
    return MEM_OK;
}

/* nsteps time steps with Alg. 3 on `nthreads` OpenMP threads (0 = the
 * OpenMP default); at most lx / 3 of them get a slab.  Needs nz >= 3 (a slab
 * of three layers) and nx, ny >= 2: case 0 leaves the first row and column
 * of a layer without a second step of their own, which holds only when
 * they are not also the last.  An odd nsteps ends with one step of Alg. 1. */
int mem_two_step_prism_omp(const mem_cfg *g, double *f, int64_t nsteps, int64_t tile, int nthreads)
{
    mem_run r;
    const int rc = setup(g, &r);
    if (rc != MEM_OK) return rc;
    if (!f || nsteps < 0 || tile < 0 || nthreads < 0 || r.lx < 3 || r.ly < 2 || r.lz < 2) return MEM_EINVAL;
    if (tile == 0) tile = r.lx + r.ly + r.lz;
#ifdef _OPENMP
    if (nthreads == 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
#ifdef MEM_CHECK
    if (chk_begin(&r) != MEM_OK) return MEM_ENOMEM;
#endif
    for (int64_t s = 0; s + 1 < nsteps; s += 2) two_step_omp(&r, f, tile, nthreads);
    if (nsteps % 2) fuse_step(&r, f);
#ifdef MEM_CHECK
    chk_end(&r, nsteps);
#endif
    return MEM_OK;
}

#ifdef MEM_CHECK
/* Checker self-test: one step of Alg. 1 with its Stage II run before Stage I,
 * so that inner cells exchange links with box cells that have not collided
 * yet; the checker must count violations.  Returns them. */
int64_t mem_check_planted_misorder(const mem_cfg *g, double *f)
{
    mem_run r;
    if (setup(g, &r) != MEM_OK || !f || chk_begin(&r) != MEM_OK) return -1;
    mem_check_reset();
    bulk_pass(&r, f);
    box_pass(&r, f, 1);
    box_pass(&r, f, 0);
    chk_end(&r, 1);
    return mem_check_violations();
}
#endif
