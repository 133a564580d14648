/*
 * cd_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the Contact
 * Dynamics (CD) time step of Shojaaee et al., "An Adaptive Hierarchical
 * Domain Decomposition Method for Parallel Contact Dynamics Simulations of
 * Granular Materials" (arXiv:1104.3516).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this code.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only
 * through the seeded input generators, which hold none of the method's
 * arithmetic.  Compile with -O2 -ffp-contract=off (no FMA contraction, no
 * fast-math) so that every floating-point operation is the one written here.
 *
 * What it computes, section by section of the paper:
 *   - contact detection, brute force and the cell method (Sec. 3.2), with the
 *     candidate distance of Eq. 12 bounded by the fixed margin delta
 *     (Sec. 3.1: l = 2.2 r_max, i.e. delta = 0.2 r_max);
 *   - contact geometry: normal n, gap g (Sec. 2.1, Fig. 1) and the pair mass
 *     matrix M built from masses and moments of inertia (Eq. 5);
 *   - the single-contact force calculation of Fig. 2: new gap with R = 0
 *     (Eq. 3), sticking force (Eqs. 4-5), Coulomb test (Eqs. 6-8) and the
 *     sliding force (Eqs. 9-11), written in impulses P = R dt;
 *   - the iterative nonlinear Gauss-Seidel over the contact network
 *     (Sec. 2.1): random sequential order re-drawn every sweep, a fixed
 *     order, or the colour order used by the GPU (greedy colouring of the
 *     contact graph with a Kempe-chain repair of its highest colour; not in
 *     the paper, a definition the GPU must reproduce); the mixed parallel /
 *     sequential update with parallelness p (Sec. 2.3); the domain-wise
 *     update of the parallel algorithm (Sec. 3.1), where every domain sweeps
 *     its own contacts while the other domains' contacts keep the impulses
 *     of the previous sweep;
 *   - the convergence tests (I) local and (II) global (Sec. 2.1, alpha);
 *   - the first-order Euler time step, Eqs. 1-2.
 *
 * Readings of passages the paper leaves open (each listed in the design
 * notes of the repository):
 *   - 2D discs carry areal mass; the mass matrix for discs and spheres is
 *     diagonal in the (n, t) frame with w_n = 1/m_a + 1/m_b and
 *     w_t = w_n + r_a^2/I_a + r_b^2/I_b (rigid-body mechanics; the paper
 *     defers M to its reference [Brendel04]).
 *   - R_avg is the mean of the impulse magnitudes |P|.
 *   - criterion ORA_CRIT_GLOBAL_REL (default) tests the non-squared relative
 *     change of R_avg against alpha; ORA_CRIT_GLOBAL_SQ is the paper's
 *     squared form (II); ORA_CRIT_LOCAL is test (I).  Both averages zero
 *     (0/0) counts as converged; a NaN average (a diverged iteration) gives
 *     a NaN ratio, which never passes.
 *   - warm start: impulses are carried over by contact key from the previous
 *     time step (off: the iteration starts from zero forces).
 *   - domain-wise update: domains are a grid of equal slabs of the box (the
 *     paper's domains come from its load balancer, out of scope here); a
 *     contact is native to the domain of the middle of its gap (Sec. 3.1);
 *     a domain sees the sweep-start velocities changed by its own updates,
 *     and the changes of all domains are summed at the end of the sweep.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_MAX_WALLS 6

enum { ORA_CRIT_NONE = -1, ORA_CRIT_GLOBAL_REL = 0, ORA_CRIT_GLOBAL_SQ = 1, ORA_CRIT_LOCAL = 2 };
enum { ORA_ORDER_COLOUR = 0, ORA_ORDER_RANDOM = 1, ORA_ORDER_FIXED = 2 };

/* Every field is 8 bytes wide so the layout has no padding surprises. */
typedef struct {
    int64_t dim;            /* 2 (discs) or 3 (spheres) */
    double dt;              /* time step */
    double mu;              /* Coulomb friction coefficient */
    double gravity[3];      /* external acceleration, treated explicitly */
    double box_lo[3];       /* box used by the cell grid and periodic wrap */
    double box_hi[3];
    int64_t periodic[3];    /* 1: periodic along that axis */
    int64_t wall_mask;      /* bit k: wall k present; k = 2*axis + side */
    double wall_vel[18];    /* kinematic wall velocities, 3 per wall */
    double delta;           /* detection margin: contact iff gap < delta */
    double alpha;           /* convergence threshold */
    int64_t criterion;      /* ORA_CRIT_* */
    int64_t max_sweeps;     /* iteration cap N_I */
    int64_t order;          /* ORA_ORDER_* */
    int64_t warm_start;     /* 1: carry impulses over by contact key */
    uint64_t seed;          /* seeds the random order and the colouring */
    double parallel_p;      /* fraction of contacts updated in parallel */
    int64_t rotations;      /* 0: rotational degrees of freedom frozen */
    double wall_push[6];    /* external force pushing wall k along its inward normal */
    double wall_mass[6];    /* > 0: wall k is a rigid body of this mass moving along
                               its normal (force-controlled); 0: kinematic */
    int64_t domains[3];     /* domain-wise update of Sec. 3.1: the box is cut
                               into domains[k] equal slabs along axis k (<= 1:
                               one); 1 x 1 x 1 is plain Gauss-Seidel */
    int64_t parallel_redraw;/* mixed update: 0 the parallel subset is fixed per
                               contact key; 1 it is drawn afresh in every
                               iteration step (see is_parallel) */
} ora_params;

/* A force-controlled wall: present, with a positive mass. */
static int wall_dynamic(const ora_params* p, int k)
{
    return (int)((p->wall_mask >> k) & 1) && (k / 2) < (int)p->dim && p->wall_mass[k] > 0.0;
}

static int64_t dyn_wall_mask(const ora_params* p)
{
    int64_t m = 0;
    for (int k = 0; k < 6; ++k) if (wall_dynamic(p, k)) m |= (int64_t)1 << k;
    return m;
}

typedef struct {
    int64_t sweeps;
    int64_t converged;
    double residual;        /* value of the chosen criterion at the last sweep */
    double r_avg;           /* R_avg (mean |P|) after the last sweep */
    double r_avg_prev;
    int64_t n_colours;
    double wall_force[ORA_MAX_WALLS];  /* sum of normal impulses / dt per wall */
} ora_solve_stats;

/* ------------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea and Flood, OOPSLA 2014), written from its        */
/* published definition: add the golden-ratio increment, then mix.          */
/* ------------------------------------------------------------------------ */
uint64_t ora_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t key_of(int32_t a, int32_t b)
{
    return ((uint64_t)(uint32_t)a << 32) | (uint64_t)(uint32_t)b;
}

/* ------------------------------------------------------------------------ */
/* Contact detection (Sec. 3.2; margin from Eq. 12 and l = 2.2 r_max)       */
/* ------------------------------------------------------------------------ */

/* Separation b - a along one axis with the minimum-image rule for a
 * periodic axis. */
static double sep_axis(const ora_params* p, int k, double xa, double xb)
{
    double d = xb - xa;
    if (p->periodic[k]) {
        double L = p->box_hi[k] - p->box_lo[k];
        if (d > 0.5 * L) d = d - L;
        else if (d < -0.5 * L) d = d + L;
    }
    return d;
}

/* Pair test: centre distance squared below (r_a + r_b + delta)^2. */
static int pair_touches(const ora_params* p, const double* x, const double* r, long long a, long long b)
{
    int D = (int)p->dim;
    double d2 = 0.0;
    for (int k = 0; k < D; ++k) {
        double d = sep_axis(p, k, x[a * D + k], x[b * D + k]);
        double dd = d * d;
        d2 = (k == 0) ? dd : d2 + dd;
    }
    double s = (r[a] + r[b]) + p->delta;
    return d2 < s * s;
}

/* Gap between particle a and wall k (plane position wall_pos[k]). */
static double wall_gap(const ora_params* p, const double* x, const double* r, const double* wall_pos, long long a, int k)
{
    int D = (int)p->dim;
    int axis = k / 2;
    double xa = x[a * D + axis];
    if ((k & 1) == 0) return (xa - wall_pos[k]) - r[a];
    return (wall_pos[k] - xa) - r[a];
}

static int wall_active(const ora_params* p, int k)
{
    return (int)((p->wall_mask >> k) & 1) && (k / 2) < (int)p->dim;
}

/* Brute force over all pairs a < b, then all walls of each particle.
 * Output sorted by key (a, b); walls have ids n + k.  Returns the number of
 * contacts found; only the first `cap` are written. */
long long ora_detect_brute(const ora_params* p, long long n, const double* x, const double* r,
                           const double* wall_pos, long long cap, int32_t* pairs)
{
    long long nc = 0;
    for (long long a = 0; a < n; ++a) {
        for (long long b = a + 1; b < n; ++b) {
            if (pair_touches(p, x, r, a, b)) {
                if (nc < cap) { pairs[2 * nc] = (int32_t)a; pairs[2 * nc + 1] = (int32_t)b; }
                ++nc;
            }
        }
        for (int k = 0; k < ORA_MAX_WALLS; ++k) {
            if (!wall_active(p, k)) continue;
            if (wall_gap(p, x, r, wall_pos, a, k) < p->delta) {
                if (nc < cap) { pairs[2 * nc] = (int32_t)a; pairs[2 * nc + 1] = (int32_t)(n + k); }
                ++nc;
            }
        }
    }
    return nc;
}

static int cmp_i32(const void* u, const void* v)
{
    int32_t a = *(const int32_t*)u, b = *(const int32_t*)v;
    return (a > b) - (a < b);
}

/* Cell method (Sec. 3.2): a grid with cell side at least l = 2 r_max + delta;
 * each particle is binned by position and only its own and the neighbouring
 * cells are searched.  Must return exactly the brute-force set. */
long long ora_detect_cells(const ora_params* p, long long n, const double* x, const double* r,
                           const double* wall_pos, long long cap, int32_t* pairs)
{
    int D = (int)p->dim;
    double rmax = 0.0;
    for (long long i = 0; i < n; ++i) if (r[i] > rmax) rmax = r[i];
    double ell = 2.0 * rmax + p->delta;
    long long nce[3] = {1, 1, 1};
    double cs[3] = {1.0, 1.0, 1.0};
    for (int k = 0; k < D; ++k) {
        double L = p->box_hi[k] - p->box_lo[k];
        long long m = (long long)floor(L / ell);
        if (m < 1) m = 1;
        nce[k] = m;
        cs[k] = L / (double)m;
    }
    long long ncell = nce[0] * nce[1] * nce[2];
    long long* head = (long long*)malloc(sizeof(long long) * (size_t)ncell);
    long long* next = (long long*)malloc(sizeof(long long) * (size_t)(n > 0 ? n : 1));
    long long* cell = (long long*)malloc(sizeof(long long) * (size_t)(n > 0 ? n : 1) * 3);
    for (long long c = 0; c < ncell; ++c) head[c] = -1;
    for (long long i = n - 1; i >= 0; --i) {
        long long ci[3] = {0, 0, 0};
        for (int k = 0; k < D; ++k) {
            long long q = (long long)floor((x[i * D + k] - p->box_lo[k]) / cs[k]);
            if (q < 0) q = 0;
            if (q > nce[k] - 1) q = nce[k] - 1;
            ci[k] = q;
            cell[i * 3 + k] = q;
        }
        long long c = (ci[2] * nce[1] + ci[1]) * nce[0] + ci[0];
        next[i] = head[c];
        head[c] = i;
    }
    int32_t* found = (int32_t*)malloc(sizeof(int32_t) * 4096);
    long long nc = 0;
    for (long long a = 0; a < n; ++a) {
        int nf = 0;
        long long visited[27];
        int nvis = 0;
        int lo2 = (D == 3) ? -1 : 0, hi2 = (D == 3) ? 1 : 0;
        for (int dz = lo2; dz <= hi2; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            long long off[3] = {dx, dy, dz};
            long long q[3] = {0, 0, 0};
            int skip = 0;
            for (int k = 0; k < D; ++k) {
                long long t = cell[a * 3 + k] + off[k];
                if (t < 0 || t >= nce[k]) {
                    if (p->periodic[k]) t = (t + nce[k]) % nce[k];
                    else skip = 1;
                }
                q[k] = t;
            }
            if (skip) continue;
            long long c = (q[2] * nce[1] + q[1]) * nce[0] + q[0];
            int dup = 0;
            for (int v = 0; v < nvis; ++v) if (visited[v] == c) dup = 1;
            if (dup) continue;
            visited[nvis++] = c;
            for (long long b = head[c]; b >= 0; b = next[b]) {
                if (b <= a) continue;
                if (pair_touches(p, x, r, a, b) && nf < 4096) found[nf++] = (int32_t)b;
            }
        }
        qsort(found, (size_t)nf, sizeof(int32_t), cmp_i32);
        for (int f = 0; f < nf; ++f) {
            if (nc < cap) { pairs[2 * nc] = (int32_t)a; pairs[2 * nc + 1] = found[f]; }
            ++nc;
        }
        for (int k = 0; k < ORA_MAX_WALLS; ++k) {
            if (!wall_active(p, k)) continue;
            if (wall_gap(p, x, r, wall_pos, a, k) < p->delta) {
                if (nc < cap) { pairs[2 * nc] = (int32_t)a; pairs[2 * nc + 1] = (int32_t)(n + k); }
                ++nc;
            }
        }
    }
    free(found); free(cell); free(next); free(head);
    return nc;
}

/* ------------------------------------------------------------------------ */
/* Contact geometry (Sec. 2.1, Fig. 1) and the pair mass matrix (Eq. 5).     */
/* n points from body a to body b; g is the surface gap.                    */
/* normal has 3 slots per contact (the third is 0 in 2D).                   */
/* ------------------------------------------------------------------------ */
void ora_contact_geometry(const ora_params* p, long long n, const double* x, const double* r,
                          const double* inv_m, const double* inv_I, const double* wall_pos,
                          long long nc, const int32_t* pairs,
                          double* normal, double* gap, double* mn, double* mt)
{
    int D = (int)p->dim;
    for (long long c = 0; c < nc; ++c) {
        long long a = pairs[2 * c], b = pairs[2 * c + 1];
        double nv[3] = {0.0, 0.0, 0.0};
        double g;
        double wa_m = inv_m[a], wa_I = p->rotations ? inv_I[a] : 0.0, ra = r[a];
        double wb_m = 0.0, wb_I = 0.0, rb = 0.0;
        if (b < n) {
            double dvec[3] = {0.0, 0.0, 0.0};
            double d2 = 0.0;
            for (int k = 0; k < D; ++k) {
                dvec[k] = sep_axis(p, k, x[a * D + k], x[b * D + k]);
                double dd = dvec[k] * dvec[k];
                d2 = (k == 0) ? dd : d2 + dd;
            }
            double d = sqrt(d2);
            if (d > 0.0) { for (int k = 0; k < D; ++k) nv[k] = dvec[k] / d; }
            else nv[0] = 1.0;   /* coincident centres: arbitrary direction */
            g = d - (r[a] + r[b]);
            wb_m = inv_m[b]; wb_I = p->rotations ? inv_I[b] : 0.0; rb = r[b];
        } else {
            int k = (int)(b - n);
            int axis = k / 2;
            nv[axis] = (k & 1) ? 1.0 : -1.0;   /* from the particle into the wall */
            g = wall_gap(p, x, r, wall_pos, a, k);
            /* a force-controlled wall moves along its normal only: it adds
             * its inverse mass to the normal row, nothing to the tangential */
            if (wall_dynamic(p, k)) wb_m = 1.0 / p->wall_mass[k];
        }
        double w_n = wa_m + wb_m;
        double w_t = (((b < n) ? w_n : wa_m) + ra * ra * wa_I) + rb * rb * wb_I;
        for (int k = 0; k < 3; ++k) normal[c * 3 + k] = nv[k];
        gap[c] = g;
        mn[c] = (w_n > 0.0) ? 1.0 / w_n : 0.0;
        mt[c] = (w_t > 0.0) ? 1.0 / w_t : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Colouring of the contact graph: two contacts conflict when they share a  */
/* particle (walls are kinematic and never conflict).  Greedy in descending */
/* priority, ties by ascending key; each contact takes the smallest colour  */
/* not used by an earlier neighbour.  prio = (d_a + d_b) * 2^56 +           */
/* (splitmix64(seed ^ key) >> 8), d = contacts of a particle (walls 0),     */
/* the sum capped at 255: largest degree first, random among equals.        */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t prio; uint64_t key; long long idx; } prio_item;

static int cmp_prio(const void* u, const void* v)
{
    const prio_item* a = (const prio_item*)u;
    const prio_item* b = (const prio_item*)v;
    if (a->prio != b->prio) return (a->prio > b->prio) ? -1 : 1;
    if (a->key != b->key) return (a->key < b->key) ? -1 : 1;
    return 0;
}

static int colour_greedy_in(long long n, long long nc, const int32_t* pairs, uint64_t seed,
                            int64_t dyn_walls, int32_t* colour);
int ora_colour_repair(long long n, long long nc, const int32_t* pairs, int64_t dyn_walls, int32_t* colour);

/* dyn_walls: bit k set when wall k is a force-controlled body, whose
 * contacts then conflict with each other like those of a particle.  The
 * greedy colouring is followed by the repair of its highest colour
 * (ora_colour_repair). */
int ora_colour_greedy(long long n, long long nc, const int32_t* pairs, uint64_t seed, int64_t dyn_walls,
                      int32_t* colour)
{
    colour_greedy_in(n, nc, pairs, seed, dyn_walls, colour);
    return ora_colour_repair(n, nc, pairs, dyn_walls, colour);
}

/* ------------------------------------------------------------------------ */
/* Repair of the highest colour by Kempe chains (the recolouring step of    */
/* the classical proof of Vizing's theorem, used here as a heuristic).  Let */
/* T be the highest colour and D the largest number of contacts of one      */
/* body.  If T + 1 > D (a colour more than any body needs) and colour T     */
/* holds at most max(1, min(1024, nc / 256)) contacts, those contacts are   */
/* visited one by one in ascending key order.  For contact c = (u, v), let  */
/* M(x) be the colours below T that no other contact of body x has (all of */
/* them for a wall that is not a body).  If M(u) and M(v) share a colour, c */
/* takes the smallest.  Otherwise, for a in M(u) and then b in M(v), both   */
/* ascending: follow from v the path whose contacts alternate colours a, b, */
/* starting with v's contact of colour a, until a body has no contact of    */
/* the next colour or the path reaches a wall; if the path reaches u, try   */
/* the next pair; else swap a and b along it (the colouring stays proper    */
/* and a is now free at v) and give c colour a.  A contact for which no     */
/* pair works keeps colour T.  Returns the number of colours afterwards.    */
/* ------------------------------------------------------------------------ */
int ora_colour_repair(long long n, long long nc, const int32_t* pairs, int64_t dyn_walls, int32_t* colour)
{
    if (nc <= 0) return 0;
#define CONFLICTS(q) ((q) < n || ((dyn_walls >> ((q) - n)) & 1))
    int kmax = 0;
    for (long long c = 0; c < nc; ++c) if (colour[c] + 1 > kmax) kmax = colour[c] + 1;
    const int T = kmax - 1;
    if (T <= 0 || T > 63) return kmax;
    const long long nb = n + 6;
    long long* deg = (long long*)calloc((size_t)nb + 1, sizeof(long long));
    for (long long c = 0; c < nc; ++c)
        for (int s = 0; s < 2; ++s) {
            long long q = pairs[2 * c + s];
            if (CONFLICTS(q)) deg[q + 1]++;
        }
    long long dmax = 0;
    for (long long i = 0; i < nb; ++i) if (deg[i + 1] > dmax) dmax = deg[i + 1];
    long long top = 0;
    for (long long c = 0; c < nc; ++c) top += (colour[c] == T);
    long long limit = nc / 256;
    if (limit > 1024) limit = 1024;
    if (limit < 1) limit = 1;
    if ((long long)kmax <= dmax || top > limit) { free(deg); return kmax; }
    for (long long i = 0; i < nb; ++i) deg[i + 1] += deg[i];
    long long* fill = (long long*)calloc((size_t)nb, sizeof(long long));
    long long* adj = (long long*)malloc(sizeof(long long) * (size_t)(deg[nb] > 0 ? deg[nb] : 1));
    for (long long c = 0; c < nc; ++c)
        for (int s = 0; s < 2; ++s) {
            long long q = pairs[2 * c + s];
            if (CONFLICTS(q)) adj[deg[q] + fill[q]++] = c;
        }
    long long* path = (long long*)malloc(sizeof(long long) * (size_t)nc);
    const uint64_t below = (1ULL << T) - 1ULL;
    for (long long c = 0; c < nc; ++c) {
        if (colour[c] != T) continue;
        const long long u = pairs[2 * c], v = pairs[2 * c + 1];
        uint64_t mu = below, mv = below;
        for (long long e = deg[u]; e < deg[u + 1]; ++e)
            if (adj[e] != c && colour[adj[e]] < T) mu &= ~(1ULL << colour[adj[e]]);
        if (CONFLICTS(v))
            for (long long e = deg[v]; e < deg[v + 1]; ++e)
                if (adj[e] != c && colour[adj[e]] < T) mv &= ~(1ULL << colour[adj[e]]);
        if (mu & mv) {
            int k = 0;
            while (!((mu & mv) >> k & 1ULL)) ++k;
            colour[c] = k;
            continue;
        }
        if (!CONFLICTS(v)) continue;
        int done = 0;
        for (int a = 0; a < T && !done; ++a) {
            if (!(mu >> a & 1ULL)) continue;
            for (int b = 0; b < T && !done; ++b) {
                if (!(mv >> b & 1ULL)) continue;
                long long len = 0, x = v;
                int cur = a, fail = 0;
                for (;;) {
                    long long e = -1;
                    for (long long f = deg[x]; f < deg[x + 1]; ++f)
                        if (colour[adj[f]] == cur) { e = adj[f]; break; }
                    if (e < 0) break;
                    long long y = (pairs[2 * e] == x) ? pairs[2 * e + 1] : pairs[2 * e];
                    path[len++] = e;
                    if (y == u) { fail = 1; break; }
                    if (!CONFLICTS(y)) break;
                    x = y;
                    cur = (cur == a) ? b : a;
                    if (len >= nc) { fail = 1; break; }
                }
                if (fail) continue;
                for (long long i = 0; i < len; ++i) colour[path[i]] = (colour[path[i]] == a) ? b : a;
                colour[c] = a;
                done = 1;
            }
        }
    }
    kmax = 0;
    for (long long c = 0; c < nc; ++c) if (colour[c] + 1 > kmax) kmax = colour[c] + 1;
    free(path); free(adj); free(fill); free(deg);
    return kmax;
#undef CONFLICTS
}

/* Greedy colouring as above: two contacts conflict when they share a particle
 * (or a force-controlled wall). */
static int colour_greedy_in(long long n, long long nc, const int32_t* pairs, uint64_t seed,
                            int64_t dyn_walls, int32_t* colour)
{
    if (nc == 0) return 0;
    /* bodies that create conflicts: the particles and the force-controlled walls n + k */
    const long long nb = n + 6;
#define CONFLICTS(q) ((q) < n || ((dyn_walls >> ((q) - n)) & 1))
    long long* deg = (long long*)calloc((size_t)nb + 1, sizeof(long long));
    for (long long c = 0; c < nc; ++c) {
        for (int s = 0; s < 2; ++s) {
            long long q = pairs[2 * c + s];
            if (CONFLICTS(q)) deg[q + 1]++;
        }
    }
    for (long long i = 0; i < nb; ++i) deg[i + 1] += deg[i];
    long long* fill = (long long*)calloc((size_t)nb + 1, sizeof(long long));
    long long* adj = (long long*)malloc(sizeof(long long) * (size_t)(deg[nb] > 0 ? deg[nb] : 1));
    for (long long c = 0; c < nc; ++c) {
        for (int s = 0; s < 2; ++s) {
            long long q = pairs[2 * c + s];
            if (CONFLICTS(q)) adj[deg[q] + fill[q]++] = c;
        }
    }
    prio_item* it = (prio_item*)malloc(sizeof(prio_item) * (size_t)nc);
    for (long long c = 0; c < nc; ++c) {
        uint64_t k = key_of(pairs[2 * c], pairs[2 * c + 1]);
        /* largest degree first: contacts per particle of both ends, summed
         * (capped at 255), in the top byte; the hash below it */
        uint64_t ds = 0;
        for (int s = 0; s < 2; ++s) {
            long long q = pairs[2 * c + s];
            if (CONFLICTS(q)) ds += (uint64_t)(deg[q + 1] - deg[q]);
        }
        if (ds > 255) ds = 255;
        it[c].prio = (ds << 56) | (ora_splitmix64(seed ^ k) >> 8);
        it[c].key = k;
        it[c].idx = c;
        colour[c] = -1;
    }
    qsort(it, (size_t)nc, sizeof(prio_item), cmp_prio);
    int kmax = 0;
    int cap = 64;
    char* used = (char*)malloc((size_t)cap);
    for (long long o = 0; o < nc; ++o) {
        long long c = it[o].idx;
        memset(used, 0, (size_t)cap);
        for (int s = 0; s < 2; ++s) {
            long long q = pairs[2 * c + s];
            if (!CONFLICTS(q)) continue;
            for (long long e = deg[q]; e < deg[q + 1]; ++e) {
                long long d = adj[e];
                if (d == c || colour[d] < 0) continue;
                if (colour[d] >= cap) {
                    int ncap = cap * 2;
                    while (ncap <= colour[d]) ncap *= 2;
                    used = (char*)realloc(used, (size_t)ncap);
                    memset(used + cap, 0, (size_t)(ncap - cap));
                    cap = ncap;
                }
                used[colour[d]] = 1;
            }
        }
        int k = 0;
        while (k < cap && used[k]) ++k;
        colour[c] = k;
        if (k + 1 > kmax) kmax = k + 1;
        if (kmax >= cap) {
            used = (char*)realloc(used, (size_t)cap * 2);
            cap *= 2;
        }
    }
    free(used); free(it); free(adj); free(fill); free(deg);
    return kmax;
#undef CONFLICTS
}

/* ------------------------------------------------------------------------ */
/* Gauss-Seidel contact solve (Sec. 2.1, Fig. 2; Sec. 2.3 for p > 0)        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const ora_params* p;
    long long n;
    double* v;        /* n*D current velocities */
    double* w;        /* n (2D) or n*3 (3D) current angular velocities */
    const double* r;
    const double* inv_m;
    const double* inv_I;
    const int32_t* pairs;
    const double* normal;
    const double* gap;
    const double* mn;
    const double* mt;
    double* wall_vel;       /* 18: wall velocities (force-controlled ones change) */
    double wall_im[6];      /* inverse mass of a force-controlled wall, else 0 */
} solve_ctx;

static int pw_of(int D) { return D == 2 ? 2 : 4; }

/* Body data: walls are bodies with infinite mass and prescribed velocity. */
static void body(const solve_ctx* s, long long q, double vq[3], double wq[3], double* rq, double* im, double* iI)
{
    int D = (int)s->p->dim;
    vq[0] = vq[1] = vq[2] = 0.0;
    wq[0] = wq[1] = wq[2] = 0.0;
    if (q < s->n) {
        for (int k = 0; k < D; ++k) vq[k] = s->v[q * D + k];
        if (D == 2) wq[2] = s->w[q];
        else for (int k = 0; k < 3; ++k) wq[k] = s->w[q * 3 + k];
        *rq = s->r[q];
        *im = s->inv_m[q];
        *iI = s->p->rotations ? s->inv_I[q] : 0.0;
    } else {
        int k = (int)(q - s->n);
        for (int j = 0; j < D; ++j) vq[j] = s->wall_vel[k * 3 + j];
        *rq = 0.0; *im = s->wall_im[k]; *iI = 0.0;
    }
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Relative velocity of the closest surface points, v_g = v_b(pt) - v_a(pt),
 * where a's point sits at +r_a n from its centre and b's at -r_b n. */
static void contact_velocity(const solve_ctx* s, long long c, double vg[3])
{
    long long a = s->pairs[2 * c], b = s->pairs[2 * c + 1];
    double va[3], wa[3], vb[3], wb[3], ra, rb, ima, imb, iIa, iIb;
    body(s, a, va, wa, &ra, &ima, &iIa);
    body(s, b, vb, wb, &rb, &imb, &iIb);
    const double* n = s->normal + c * 3;
    double la[3] = {ra * n[0], ra * n[1], ra * n[2]};
    double lb[3] = {-rb * n[0], -rb * n[1], -rb * n[2]};
    double ca[3], cb[3];
    cross3(wa, la, ca);
    cross3(wb, lb, cb);
    for (int k = 0; k < 3; ++k) vg[k] = (vb[k] + cb[k]) - (va[k] + ca[k]);
}

/* Impulse change dP (global vector) acts +dP on b and -dP on a, each at its
 * contact point. */
static void apply_impulse(solve_ctx* s, long long c, const double dP[3])
{
    int D = (int)s->p->dim;
    const double* n = s->normal + c * 3;
    for (int side = 0; side < 2; ++side) {
        long long q = s->pairs[2 * c + side];
        double sign = side ? 1.0 : -1.0;
        if (q >= s->n) {
            /* a force-controlled wall takes the impulse along its normal */
            int k = (int)(q - s->n);
            if (s->wall_im[k] > 0.0) s->wall_vel[k * 3 + k / 2] += sign * s->wall_im[k] * dP[k / 2];
            continue;
        }
        double im = s->inv_m[q];
        double iI = s->p->rotations ? s->inv_I[q] : 0.0;
        double rq = s->r[q];
        for (int k = 0; k < D; ++k) s->v[q * D + k] += sign * im * dP[k];
        /* torque arm: +r n for a, -r n for b; torque = arm x (sign dP) */
        double arm[3] = {(side ? -rq : rq) * n[0], (side ? -rq : rq) * n[1], (side ? -rq : rq) * n[2]};
        double f[3] = {sign * dP[0], sign * dP[1], sign * dP[2]};
        double tq[3];
        cross3(arm, f, tq);
        if (D == 2) s->w[q] += iI * tq[2];
        else for (int k = 0; k < 3; ++k) s->w[q * 3 + k] += iI * tq[k];
    }
}

/* Global impulse vector of contact c from its stored components.
 * 2D: P = (Pn, Pt) in the (n, t) frame, t = (-n_y, n_x).
 * 3D: P = (Pn, Ptx, Pty, Ptz), the tangential part as a global vector. */
static void impulse_vector(int D, const double* n, const double* Pc, double out[3])
{
    if (D == 2) {
        out[0] = Pc[0] * n[0] - Pc[1] * n[1];
        out[1] = Pc[0] * n[1] + Pc[1] * n[0];
        out[2] = 0.0;
    } else {
        for (int k = 0; k < 3; ++k) out[k] = Pc[0] * n[k] + Pc[1 + k];
    }
}

/* Fig. 2: the force calculation for a single contact, given that all other
 * forces on its two bodies are known (they are folded into v, w).  Pc is
 * updated in place and the change is applied to the bodies.  If dP_out is
 * non-NULL the change is returned instead of applied (parallel update). */
static void solve_one(solve_ctx* s, long long c, double* Pc, double* dP_out)
{
    const ora_params* p = s->p;
    int D = (int)p->dim;
    const double* n = s->normal + c * 3;
    double dt = p->dt;
    double mn = s->mn[c], mt = s->mt[c];
    /* M^-1 of the pair (the inverse of the mass matrix of Eq. 5) */
    double va_[3], wa_[3], vb_[3], wb_[3], ra, rb, ima, imb, iIa, iIb;
    body(s, s->pairs[2 * c], va_, wa_, &ra, &ima, &iIa);
    body(s, s->pairs[2 * c + 1], vb_, wb_, &rb, &imb, &iIb);
    double wn = ima + imb;
    /* a wall moves along its normal only: no share in the tangential row */
    double wt = (((s->pairs[2 * c + 1] < s->n) ? wn : ima) + ra * ra * iIa) + rb * rb * iIb;
    double vg[3];
    contact_velocity(s, c, vg);
    double Pnew[4] = {0.0, 0.0, 0.0, 0.0};
    if (D == 2) {
        double t[2] = {-n[1], n[0]};
        double vn = vg[0] * n[0] + vg[1] * n[1];
        double vt = vg[0] * t[0] + vg[1] * t[1];
        /* relative velocity without this contact's own impulse (v_g0) */
        double v0n = vn - wn * Pc[0];
        double v0t = vt - wt * Pc[1];
        /* Eq. 3: new gap assuming R = 0 */
        double gnew = s->gap[c] + v0n * dt;
        if (gnew > 0.0) {
            Pnew[0] = 0.0; Pnew[1] = 0.0;
        } else {
            /* Eq. 5, sticking: P = -M (g/dt n + v_g0) */
            double Pn = -mn * (s->gap[c] / dt + v0n);
            double Pt = -mt * v0t;
            /* Eq. 8: Coulomb cone; otherwise sliding, Eqs. 9-11 */
            if (fabs(Pt) > p->mu * Pn) {
                double sgn = (v0t > 0.0) ? 1.0 : -1.0;
                Pt = -p->mu * Pn * sgn;
            }
            Pnew[0] = Pn; Pnew[1] = Pt;
        }
    } else {
        double vn = vg[0] * n[0] + vg[1] * n[1] + vg[2] * n[2];
        double vt[3];
        for (int k = 0; k < 3; ++k) vt[k] = vg[k] - vn * n[k];
        double v0n = vn - wn * Pc[0];
        double v0t[3];
        for (int k = 0; k < 3; ++k) v0t[k] = vt[k] - wt * Pc[1 + k];
        double gnew = s->gap[c] + v0n * dt;
        if (gnew > 0.0) {
            for (int k = 0; k < 4; ++k) Pnew[k] = 0.0;
        } else {
            double Pn = -mn * (s->gap[c] / dt + v0n);
            double Pt[3];
            for (int k = 0; k < 3; ++k) Pt[k] = -mt * v0t[k];
            double ptn = sqrt(Pt[0] * Pt[0] + Pt[1] * Pt[1] + Pt[2] * Pt[2]);
            if (ptn > p->mu * Pn) {
                /* sliding against the tangential relative velocity */
                double un = sqrt(v0t[0] * v0t[0] + v0t[1] * v0t[1] + v0t[2] * v0t[2]);
                for (int k = 0; k < 3; ++k) Pt[k] = -p->mu * Pn * (v0t[k] / un);
            }
            Pnew[0] = Pn; Pnew[1] = Pt[0]; Pnew[2] = Pt[1]; Pnew[3] = Pt[2];
        }
    }
    int pw = pw_of(D);
    double dPc[4];
    for (int k = 0; k < pw; ++k) dPc[k] = Pnew[k] - Pc[k];
    double dP[3];
    impulse_vector(D, n, dPc, dP);
    if (dP_out) {
        for (int k = 0; k < 3; ++k) dP_out[k] = dP[k];
    } else {
        apply_impulse(s, c, dP);
    }
    for (int k = 0; k < pw; ++k) Pc[k] = Pnew[k];
}

static double impulse_norm(int D, const double* Pc)
{
    if (D == 2) return sqrt(Pc[0] * Pc[0] + Pc[1] * Pc[1]);
    return sqrt(Pc[0] * Pc[0] + Pc[1] * Pc[1] + Pc[2] * Pc[2] + Pc[3] * Pc[3]);
}

/* Uniform index in [0, m) from a splitmix64 counter stream. */
static uint64_t rng_next(uint64_t* state)
{
    *state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* Domain-wise update (Sec. 3.1).  The box is cut into a grid of equal      */
/* domains; a contact belongs to the domain holding its position, the       */
/* middle of the gap between the two surfaces: q = x_a + n (r_a + g / 2)    */
/* (a wall contact likewise, n pointing from the particle into the wall),   */
/* wrapped on a periodic axis.  Slab index along axis k:                    */
/* floor(((q - lo) / (hi - lo)) * domains[k]), clamped; domain id = ix +     */
/* nx (iy + ny iz).  Returns the number of domains.                         */
/* ------------------------------------------------------------------------ */
static int64_t n_domains_axis(const ora_params* p, int k)
{
    return (k < (int)p->dim && p->domains[k] > 1) ? p->domains[k] : 1;
}

int64_t ora_contact_domains(const ora_params* p, long long n, const double* x, const double* r, long long nc,
                            const int32_t* pairs, const double* normal, const double* gap, int32_t* out)
{
    int D = (int)p->dim;
    int64_t total = 1;
    for (int k = 0; k < 3; ++k) total *= n_domains_axis(p, k);
    (void)n;
    for (long long c = 0; c < nc; ++c) {
        long long a = pairs[2 * c];
        int64_t id = 0, mult = 1;
        for (int k = 0; k < D; ++k) {
            int64_t nd = n_domains_axis(p, k);
            if (nd > 1) {
                double q = x[a * D + k] + normal[c * 3 + k] * (r[a] + 0.5 * gap[c]);
                double lo = p->box_lo[k], hi = p->box_hi[k];
                if (p->periodic[k]) {
                    if (q >= hi) q = q - (hi - lo);
                    else if (q < lo) q = q + (hi - lo);
                }
                double t = ((q - lo) / (hi - lo)) * (double)nd;
                int64_t ix = (int64_t)floor(t);
                if (ix < 0) ix = 0;
                if (ix > nd - 1) ix = nd - 1;
                id += ix * mult;
            }
            mult *= nd;
        }
        out[c] = (int32_t)id;
    }
    return total;
}

/* A contact is in the parallel-update set of Sec. 2.3 when a uniform number
 * drawn for it falls below p.  The draw is splitmix64 of the contact key
 * mixed with the seed: one fixed subset per contact key (parallel_redraw 0),
 * or, with the iteration step's number mixed in as well, a fresh subset in
 * every iteration step (parallel_redraw 1), the way the paper draws its
 * random sequential order anew each step (Sec. 2.1). */
static int is_parallel(const ora_params* p, uint64_t key, long long sweep)
{
    if (p->parallel_p <= 0.0) return 0;
    if (p->parallel_p >= 1.0) return 1;
    uint64_t x = key ^ (p->seed * 0xD1B54A32D192ED03ULL);
    if (p->parallel_redraw) x ^= (uint64_t)(sweep + 1) * 0x9E3779B97F4A7C15ULL;
    uint64_t h = ora_splitmix64(x);
    double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    return u < p->parallel_p;
}

static const int32_t* g_sort_colour;

static int cmp_colour(const void* u, const void* v)
{
    long long a = *(const long long*)u, b = *(const long long*)v;
    if (g_sort_colour[a] != g_sort_colour[b]) return (g_sort_colour[a] < g_sort_colour[b]) ? -1 : 1;
    return (a > b) - (a < b);
}

/* Solve the contact impulses of one time step: the iterative nonlinear
 * Gauss-Seidel of Sec. 2.1 over the single-contact solve of Fig. 2, in the
 * chosen order, until the convergence test (I) or (II) passes.
 *   v, w     in: free velocities (external forces applied, no contact
 *                impulses); out: velocities with the final impulses applied.
 *   P        in: starting impulses (warm start or zeros); out: solution.
 *   colour   colour per contact (ORA_ORDER_COLOUR), may be NULL otherwise.
 *   fixed    the order for ORA_ORDER_FIXED, may be NULL otherwise.
 *   domain   domain of each contact (ora_contact_domains) for the
 *            domain-wise update of Sec. 3.1, or NULL (one domain).
 *   ravg_hist  if non-NULL, R_avg after sweep j is stored at [j]
 *              ([0] = starting impulses); room for max_sweeps + 1.
 * Returns 0. */
int ora_solve(ora_params* p, long long n, double* v, double* w,
              const double* r, const double* inv_m, const double* inv_I,
              long long nc, const int32_t* pairs, const double* normal, const double* gap,
              const double* mn, const double* mt, const int32_t* colour,
              const int32_t* fixed, const int32_t* domain, long long step_index, double* P, double* ravg_hist,
              ora_solve_stats* st)
{
    int D = (int)p->dim;
    int pw = pw_of(D);
    solve_ctx s;
    s.p = p; s.n = n; s.v = v; s.w = w; s.r = r; s.inv_m = inv_m; s.inv_I = inv_I;
    s.pairs = pairs; s.normal = normal; s.gap = gap; s.mn = mn; s.mt = mt;
    double wall_vel[18];
    for (int k = 0; k < 18; ++k) wall_vel[k] = p->wall_vel[k];
    s.wall_vel = wall_vel;
    for (int k = 0; k < 6; ++k) s.wall_im[k] = wall_dynamic(p, k) ? 1.0 / p->wall_mass[k] : 0.0;
    memset(st, 0, sizeof(*st));

    /* apply the starting impulses (key order) */
    for (long long c = 0; c < nc; ++c) {
        double dP[3];
        impulse_vector(D, normal + c * 3, P + c * pw, dP);
        apply_impulse(&s, c, dP);
    }

    long long* order = (long long*)malloc(sizeof(long long) * (size_t)(nc > 0 ? nc : 1));
    if (p->order == ORA_ORDER_COLOUR) {
        /* (colour, key): a stable sort of the key-ordered contacts */
        int K = 0;
        for (long long c = 0; c < nc; ++c) if (colour[c] + 1 > K) K = colour[c] + 1;
        st->n_colours = K;
        for (long long c = 0; c < nc; ++c) order[c] = c;
        g_sort_colour = colour;
        qsort(order, (size_t)nc, sizeof(long long), cmp_colour);
    } else {
        for (long long c = 0; c < nc; ++c) order[c] = (p->order == ORA_ORDER_FIXED && fixed) ? fixed[c] : c;
    }
    char* par = (char*)malloc((size_t)(nc > 0 ? nc : 1));
    long long npar = 0;
    for (long long c = 0; c < nc; ++c) {
        /* the domain-wise update replaces the mixed update of Sec. 2.3 */
        par[c] = domain ? 0 : (char)is_parallel(p, key_of(pairs[2 * c], pairs[2 * c + 1]), 0);
        npar += par[c];
    }
    double* Pprev = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1) * (size_t)pw);
    double* dPpar = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1) * 3);
    int32_t ndom = 1;
    if (domain) for (long long c = 0; c < nc; ++c) if (domain[c] + 1 > ndom) ndom = domain[c] + 1;
    const size_t nv = (size_t)(n > 0 ? n : 1) * (size_t)D, nw = (size_t)(n > 0 ? n : 1) * (size_t)(D == 2 ? 1 : 3);
    double* v0 = (double*)malloc(sizeof(double) * nv);
    double* w0 = (double*)malloc(sizeof(double) * nw);
    double* vsum = (double*)malloc(sizeof(double) * nv);
    double* wsum = (double*)malloc(sizeof(double) * nw);

    double ravg_prev = 0.0;
    for (long long c = 0; c < nc; ++c) ravg_prev += impulse_norm(D, P + c * pw);
    if (nc > 0) ravg_prev /= (double)nc;
    if (ravg_hist) ravg_hist[0] = ravg_prev;
    st->r_avg = ravg_prev;

    long long sweep = 0;
    int converged = (nc == 0);
    double resid = 0.0;
    while (!converged && sweep < p->max_sweeps) {
        memcpy(Pprev, P, sizeof(double) * (size_t)nc * (size_t)pw);
        if (p->order == ORA_ORDER_RANDOM) {
            /* Sec. 2.1: contacts chosen randomly one by one, a fresh random
             * permutation in every iteration step (Fisher-Yates). */
            uint64_t st_rng = p->seed ^ ((uint64_t)(step_index + 1) * 0xA24BAED4963EE407ULL)
                              ^ ((uint64_t)(sweep + 1) * 0x9FB21C651E98DF25ULL);
            for (long long c = 0; c < nc; ++c) order[c] = c;
            for (long long i = nc - 1; i > 0; --i) {
                long long j = (long long)(rng_next(&st_rng) % (uint64_t)(i + 1));
                long long t = order[i]; order[i] = order[j]; order[j] = t;
            }
        }
        if (p->parallel_redraw && !domain && p->parallel_p > 0.0 && p->parallel_p < 1.0) {
            /* a fresh parallel subset for this iteration step */
            npar = 0;
            for (long long c = 0; c < nc; ++c) {
                par[c] = (char)is_parallel(p, key_of(pairs[2 * c], pairs[2 * c + 1]), sweep);
                npar += par[c];
            }
        }
        if (npar > 0) {
            /* Sec. 2.3, parallel part: computed from the values at the start
             * of the sweep, applied at its end. */
            for (long long c = 0; c < nc; ++c)
                if (par[c]) solve_one(&s, c, P + c * pw, dPpar + c * 3);
        }
        if (domain) {
            /* Sec. 3.1: every domain sweeps its own (native) contacts in the
             * sweep order, seeing the velocities of the sweep start changed
             * by its own updates only: the contacts of other domains keep
             * the impulses of the last sweep.  At the end of the sweep the
             * velocity changes of all domains are added up. */
            double u0[18], usum[18];   /* force-controlled walls: the same */
            memcpy(v0, v, sizeof(double) * nv);
            memcpy(w0, w, sizeof(double) * nw);
            memcpy(u0, wall_vel, sizeof(u0));
            memcpy(vsum, v0, sizeof(double) * nv);
            memcpy(wsum, w0, sizeof(double) * nw);
            memcpy(usum, u0, sizeof(u0));
            for (int32_t d = 0; d < ndom; ++d) {
                memcpy(v, v0, sizeof(double) * nv);
                memcpy(w, w0, sizeof(double) * nw);
                memcpy(wall_vel, u0, sizeof(u0));
                for (long long o = 0; o < nc; ++o) {
                    long long c = order[o];
                    if (domain[c] == d) solve_one(&s, c, P + c * pw, NULL);
                }
                for (size_t i = 0; i < nv; ++i) vsum[i] = vsum[i] + (v[i] - v0[i]);
                for (size_t i = 0; i < nw; ++i) wsum[i] = wsum[i] + (w[i] - w0[i]);
                for (int k = 0; k < 18; ++k) usum[k] = usum[k] + (wall_vel[k] - u0[k]);
            }
            memcpy(v, vsum, sizeof(double) * nv);
            memcpy(w, wsum, sizeof(double) * nw);
            memcpy(wall_vel, usum, sizeof(usum));
        } else {
            for (long long o = 0; o < nc; ++o) {
                long long c = order[o];
                if (par[c]) continue;
                solve_one(&s, c, P + c * pw, NULL);
            }
        }
        if (npar > 0) {
            for (long long c = 0; c < nc; ++c)
                if (par[c]) apply_impulse(&s, c, dPpar + c * 3);
        }
        ++sweep;

        /* convergence (Sec. 2.1, tests I and II) */
        double ravg = 0.0;
        for (long long c = 0; c < nc; ++c) ravg += impulse_norm(D, P + c * pw);
        ravg /= (double)nc;
        if (ravg_hist) ravg_hist[sweep] = ravg;
        double den = ravg + ravg_prev;
        if (p->criterion == ORA_CRIT_GLOBAL_REL) {
            resid = (den > 0.0) ? fabs(ravg - ravg_prev) / den : (den == 0.0 ? 0.0 : den);
            converged = resid < p->alpha;
        } else if (p->criterion == ORA_CRIT_GLOBAL_SQ) {
            double q = (den > 0.0) ? (ravg - ravg_prev) / den : (den == 0.0 ? 0.0 : den);
            resid = q * q;
            converged = resid < p->alpha;
        } else if (p->criterion == ORA_CRIT_LOCAL) {
            long long n_rel = 0, n_bad = 0;
            for (long long c = 0; c < nc; ++c) {
                double d2 = 0.0, s2 = 0.0;
                for (int k = 0; k < pw; ++k) {
                    double dk = P[c * pw + k] - Pprev[c * pw + k];
                    double sk = P[c * pw + k] + Pprev[c * pw + k];
                    d2 += dk * dk;
                    s2 += sk * sk;
                }
                if (d2 < p->alpha * s2) ++n_rel;
                else if (!(d2 <= p->alpha * ravg_prev * ravg_prev)) ++n_bad;
            }
            resid = (nc > 0) ? (double)(nc - n_rel) / (double)nc : 0.0;
            converged = (10 * n_rel >= 9 * nc) && n_bad == 0;
        } else {
            resid = (den > 0.0) ? fabs(ravg - ravg_prev) / den : (den == 0.0 ? 0.0 : den);
            converged = 0;
        }
        st->r_avg_prev = ravg_prev;
        st->r_avg = ravg;
        ravg_prev = ravg;
    }
    st->sweeps = sweep;
    st->converged = converged;
    st->residual = resid;
    for (long long c = 0; c < nc; ++c) {
        long long b = pairs[2 * c + 1];
        if (b >= n) st->wall_force[b - n] += P[c * pw] / p->dt;
    }
    for (int k = 0; k < 18; ++k) p->wall_vel[k] = wall_vel[k];   /* force-controlled walls moved */
    free(wsum); free(vsum); free(w0); free(v0);
    free(dPpar); free(Pprev); free(par); free(order);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One CD time step (Fig. 3): detection, force calculation, Euler update.   */
/* ------------------------------------------------------------------------ */
static long long find_key(long long nc, const int32_t* pairs, uint64_t k)
{
    long long lo = 0, hi = nc - 1;
    while (lo <= hi) {
        long long mid = lo + (hi - lo) / 2;
        uint64_t km = key_of(pairs[2 * mid], pairs[2 * mid + 1]);
        if (km == k) return mid;
        if (km < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* One CD time step (Fig. 3): free flight (Eq. 1), detection (Sec. 3.2),
 * warm start, ordering, the force calculation (ora_solve) and the Euler
 * update of positions and orientations (Eq. 2).
 * State arrays are updated in place.
 *   x, v: n*D; w: n (2D) or n*3 (3D); theta: n (2D orientation, may be NULL)
 *   f_ext: n*D explicit external forces (may be NULL)
 *   wall_pos: 6 plane positions, moved with the wall velocities
 *   pairs_io/P_io/nc_io: in = previous step's contacts (warm start), out =
 *   this step's contacts and impulses in key order; capacity `cap`.
 *   normal_out, gap_out (may be NULL): this step's geometry, cap*3 and cap.
 * Returns 0, or -1 if the contacts exceed `cap` (then *nc_io holds the number
 * needed and nothing is changed). */
int ora_step(ora_params* p, long long n, double* x, double* v, double* w, double* theta,
             const double* r, const double* inv_m, const double* inv_I, const double* f_ext,
             double* wall_pos, long long cap, long long* nc_io, int32_t* pairs_io, double* P_io,
             long long step_index, int use_cells, int32_t* colour_out,
             double* normal_out, double* gap_out, ora_solve_stats* st)
{
    int D = (int)p->dim;
    int pw = pw_of(D);
    int32_t* pairs = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(cap > 0 ? cap : 1));
    long long nc = use_cells ? ora_detect_cells(p, n, x, r, wall_pos, cap, pairs)
                             : ora_detect_brute(p, n, x, r, wall_pos, cap, pairs);
    if (nc > cap) { free(pairs); *nc_io = nc; return -1; }
    size_t ncz = (size_t)(nc > 0 ? nc : 1);
    double* normal = (double*)malloc(sizeof(double) * ncz * 3);
    double* gap = (double*)malloc(sizeof(double) * ncz);
    double* mn = (double*)malloc(sizeof(double) * ncz);
    double* mt = (double*)malloc(sizeof(double) * ncz);
    double* P = (double*)calloc(ncz * (size_t)pw, sizeof(double));
    int32_t* colour = (int32_t*)malloc(sizeof(int32_t) * ncz);
    ora_contact_geometry(p, n, x, r, inv_m, inv_I, wall_pos, nc, pairs, normal, gap, mn, mt);

    /* warm start by key; in 3D the old tangential impulse is projected onto
     * the new tangent plane */
    if (p->warm_start) {
        long long nprev = *nc_io;
        for (long long c = 0; c < nc; ++c) {
            long long o = find_key(nprev, pairs_io, key_of(pairs[2 * c], pairs[2 * c + 1]));
            if (o < 0) continue;
            if (D == 2) {
                P[c * 2] = P_io[o * 2];
                P[c * 2 + 1] = P_io[o * 2 + 1];
            } else {
                const double* nn = normal + c * 3;
                const double* q = P_io + o * 4;
                double tn = q[1] * nn[0] + q[2] * nn[1] + q[3] * nn[2];
                P[c * 4] = q[0];
                for (int k = 0; k < 3; ++k) P[c * 4 + 1 + k] = q[1 + k] - tn * nn[k];
            }
        }
    }

    /* free flight: explicit external forces (Eq. 1 with F = m g + f_ext) */
    for (long long i = 0; i < n; ++i) {
        for (int k = 0; k < D; ++k) {
            double a = p->gravity[k];
            if (inv_m[i] == 0.0) a = 0.0;
            if (f_ext) a = a + f_ext[i * D + k] * inv_m[i];
            v[i * D + k] = v[i * D + k] + a * p->dt;
        }
    }
    /* a force-controlled wall: its push along the inward normal, explicitly (Eq. 1) */
    for (int k = 0; k < ORA_MAX_WALLS; ++k) {
        if (!wall_dynamic(p, k)) continue;
        double a = p->wall_push[k] / p->wall_mass[k];
        if (k & 1) a = -a;
        p->wall_vel[k * 3 + k / 2] = p->wall_vel[k * 3 + k / 2] + a * p->dt;
    }

    ora_params q = *p;
    if (p->order == ORA_ORDER_COLOUR) {
        int K = ora_colour_greedy(n, nc, pairs, p->seed, dyn_wall_mask(p), colour);
        (void)K;
    } else {
        for (long long c = 0; c < nc; ++c) colour[c] = 0;
    }
    int32_t* domain = NULL;
    if (n_domains_axis(p, 0) * n_domains_axis(p, 1) * n_domains_axis(p, 2) > 1) {
        domain = (int32_t*)malloc(sizeof(int32_t) * ncz);
        ora_contact_domains(p, n, x, r, nc, pairs, normal, gap, domain);
    }
    ora_solve(&q, n, v, w, r, inv_m, inv_I, nc, pairs, normal, gap, mn, mt, colour, NULL, domain,
              step_index, P, NULL, st);
    for (int k = 0; k < 18; ++k) p->wall_vel[k] = q.wall_vel[k];
    free(domain);

    /* Eq. 2: positions with the new velocities; orientation likewise */
    for (long long i = 0; i < n; ++i) {
        for (int k = 0; k < D; ++k) {
            double xn = x[i * D + k] + v[i * D + k] * p->dt;
            if (p->periodic[k]) {
                double L = p->box_hi[k] - p->box_lo[k];
                if (xn >= p->box_hi[k]) xn = xn - L;
                else if (xn < p->box_lo[k]) xn = xn + L;
            }
            x[i * D + k] = xn;
        }
        if (D == 2 && theta) theta[i] = theta[i] + w[i] * p->dt;
    }
    for (int k = 0; k < ORA_MAX_WALLS; ++k) {
        if (!wall_active(p, k)) continue;
        wall_pos[k] = wall_pos[k] + p->wall_vel[k * 3 + k / 2] * p->dt;
    }

    memcpy(pairs_io, pairs, sizeof(int32_t) * 2 * (size_t)nc);
    memcpy(P_io, P, sizeof(double) * (size_t)nc * (size_t)pw);
    if (colour_out) memcpy(colour_out, colour, sizeof(int32_t) * (size_t)nc);
    if (normal_out) memcpy(normal_out, normal, sizeof(double) * (size_t)nc * 3);
    if (gap_out) memcpy(gap_out, gap, sizeof(double) * (size_t)nc);
    *nc_io = nc;
    free(colour); free(P); free(mt); free(mn); free(gap); free(normal); free(pairs);
    return 0;
}
