/*
 * cd_workloads.c -- seeded synthetic packings for the Contact Dynamics path.
 *
 * Input generation only: random radii, random sequential addition (RSA)
 * gases, jittered lattices and a gravity deposition of discs.  Nothing here
 * computes contact forces, impulses or any step of the CD method; both the
 * CUDA library and the CPU oracle consume these arrays unchanged.
 *
 * Randomness: splitmix64 (Steele, Lea and Flood 2014) as a counter-based
 * stream; normals by the Box-Muller transform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t sm64_next(uint64_t* s)
{
    *s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = *s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in [0, 1) with 53 random bits */
static double u01(uint64_t* s) { return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0); }

void wl_uniform(uint64_t seed, int64_t n, double lo, double hi, double* out)
{
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * u01(&s);
}

void wl_normal(uint64_t seed, int64_t n, double sigma, double* out)
{
    uint64_t s = seed;
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < n; i += 2) {
        double u1 = u01(&s), u2 = u01(&s);
        if (u1 < 1e-300) u1 = 1e-300;
        double rad = sqrt(-2.0 * log(u1));
        out[i] = sigma * rad * cos(two_pi * u2);
        if (i + 1 < n) out[i + 1] = sigma * rad * sin(two_pi * u2);
    }
}

static double min_image(double d, double L, int periodic)
{
    if (!periodic) return d;
    if (d > 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
    return d;
}

/* ------------------------------------------------------------------------ */
/* Random sequential addition in a box (2D or 3D).  Particle i is placed    */
/* with its full disc inside non-periodic extents; candidates overlapping a */
/* placed particle are rejected.  Returns the number placed.                */
/* ------------------------------------------------------------------------ */
int64_t wl_rsa(int64_t dim, int64_t n, const double* radii, const double* lo, const double* hi,
               const int64_t* periodic, double min_gap, uint64_t seed, int64_t max_attempts, double* x)
{
    int D = (int)dim;
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (radii[i] > rmax) rmax = radii[i];
    double cs_min = 2.0 * rmax + min_gap;
    int64_t nce[3] = {1, 1, 1};
    double cs[3] = {1, 1, 1}, L[3] = {1, 1, 1};
    for (int k = 0; k < D; ++k) {
        L[k] = hi[k] - lo[k];
        nce[k] = (int64_t)floor(L[k] / cs_min);
        if (nce[k] < 1) nce[k] = 1;
        cs[k] = L[k] / (double)nce[k];
    }
    int64_t ncell = nce[0] * nce[1] * nce[2];
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    uint64_t s = seed;
    int64_t placed = 0, attempts = 0;
    while (placed < n && attempts < max_attempts) {
        ++attempts;
        double ri = radii[placed];
        double c[3] = {0, 0, 0};
        int64_t q[3] = {0, 0, 0};
        for (int k = 0; k < D; ++k) {
            double a = lo[k], b = hi[k];
            if (!periodic[k]) { a += ri; b -= ri; }
            c[k] = a + (b - a) * u01(&s);
            int64_t t = (int64_t)floor((c[k] - lo[k]) / cs[k]);
            if (t < 0) t = 0;
            if (t >= nce[k]) t = nce[k] - 1;
            q[k] = t;
        }
        int ok = 1;
        int lz = D == 3 ? -1 : 0, hz = D == 3 ? 1 : 0;
        for (int dz = lz; dz <= hz && ok; ++dz)
        for (int dy = -1; dy <= 1 && ok; ++dy)
        for (int dx = -1; dx <= 1 && ok; ++dx) {
            int64_t off[3] = {dx, dy, dz}, cc[3] = {0, 0, 0};
            int skip = 0;
            for (int k = 0; k < D; ++k) {
                int64_t t = q[k] + off[k];
                if (t < 0 || t >= nce[k]) {
                    if (periodic[k]) t = (t + nce[k]) % nce[k]; else skip = 1;
                }
                cc[k] = t;
            }
            if (skip) continue;
            int64_t cell = (cc[2] * nce[1] + cc[1]) * nce[0] + cc[0];
            for (int64_t j = head[cell]; j >= 0; j = next[j]) {
                double d2 = 0.0;
                for (int k = 0; k < D; ++k) {
                    double d = min_image(x[j * D + k] - c[k], L[k], (int)periodic[k]);
                    d2 += d * d;
                }
                double sr = ri + radii[j] + min_gap;
                if (d2 < sr * sr) { ok = 0; break; }
            }
        }
        if (!ok) continue;
        for (int k = 0; k < D; ++k) x[placed * D + k] = c[k];
        int64_t cell = (q[2] * nce[1] + q[1]) * nce[0] + q[0];
        next[placed] = head[cell];
        head[cell] = placed;
        ++placed;
    }
    free(next); free(head);
    return placed;
}

/* ------------------------------------------------------------------------ */
/* Gravity deposition of discs (2D), after Visscher and Bolsterli (Nature   */
/* 1972): each disc is dropped at a random x, falls until it touches a      */
/* placed disc or the floor, then rolls over its support until it rests on  */
/* two supports on either side of its centre, or on the floor.  Periodic in */
/* x over [0, Lx); floor at y = 0.  Contacts are exact up to rounding.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double Lx, cs, rmax;
    int64_t ncx, ncy;
    int64_t* head;
    int64_t* next;
    int64_t* coltop;   /* highest occupied cell row per column, -1 if empty */
    double* x;         /* 2 per disc */
    const double* r;
} depo;

static int64_t col_of(const depo* d, double x)
{
    int64_t c = (int64_t)floor(x / d->cs);
    if (c < 0) c = 0;
    if (c >= d->ncx) c = d->ncx - 1;
    return c;
}

static int64_t row_of(const depo* d, double y)
{
    int64_t c = (int64_t)floor(y / d->cs);
    if (c < 0) c = 0;
    if (c >= d->ncy) c = d->ncy - 1;
    return c;
}

/* Highest y <= ycap at which disc (x, ri) falling vertically first touches a
 * disc (not `skip`) or the floor.  Returns the support id, or -1 for floor. */
static int64_t fall(const depo* d, double x, double ri, double ycap, int64_t skip, double* yout)
{
    double best = ri;  /* floor */
    int64_t who = -1;
    double reach = ri + d->rmax;
    int64_t span = (int64_t)ceil(reach / d->cs);
    int64_t c0 = col_of(d, x);
    for (int64_t dc = -span; dc <= span; ++dc) {
        int64_t c = ((c0 + dc) % d->ncx + d->ncx) % d->ncx;
        for (int64_t row = d->coltop[c]; row >= 0; --row) {
            /* any disc in this row has y < (row+1)*cs; contact height below that + reach */
            double ymax_row = (double)(row + 1) * d->cs + reach;
            if (ymax_row < best) break;
            for (int64_t j = d->head[row * d->ncx + c]; j >= 0; j = d->next[j]) {
                if (j == skip) continue;
                double dx = min_image(d->x[2 * j] - x, d->Lx, 1);
                double R = ri + d->r[j];
                if (fabs(dx) >= R) continue;
                double yc = d->x[2 * j + 1] + sqrt(R * R - dx * dx);
                if (yc > ycap) continue;
                if (yc > best) { best = yc; who = j; }
            }
        }
    }
    *yout = best;
    return who;
}

/* Roll disc i (radius ri) over support j starting at angle phi0 from the
 * vertical, on side s (+1: towards +x).  Finds the first contact with
 * another disc or the floor for phi in (phi0, pi/2].  Returns the id of the
 * disc met, -1 for the floor, -2 if none (rolled to the horizontal). */
static int64_t roll(const depo* d, double ri, int64_t j, double phi0, int s, double* phi_out)
{
    double xj = d->x[2 * j], yj = d->x[2 * j + 1];
    double R = ri + d->r[j];
    double best = 1.5707963267948966;
    int64_t who = -2;
    /* floor: yj + R cos(phi) = ri */
    double cf = (ri - yj) / R;
    if (cf > -1.0 && cf < 1.0) {
        double pf = acos(cf);
        if (pf > phi0 + 1e-12 && pf <= best) { best = pf; who = -1; }
    }
    int64_t span = (int64_t)ceil((R + ri + d->rmax) / d->cs);
    int64_t c0 = col_of(d, xj), r0 = row_of(d, yj);
    for (int64_t dr = -span; dr <= span; ++dr) {
        int64_t row = r0 + dr;
        if (row < 0 || row >= d->ncy) continue;
        for (int64_t dc = -span; dc <= span; ++dc) {
            int64_t c = ((c0 + dc) % d->ncx + d->ncx) % d->ncx;
            for (int64_t k = d->head[row * d->ncx + c]; k >= 0; k = d->next[k]) {
                if (k == j) continue;
                double ex = min_image(d->x[2 * k] - xj, d->Lx, 1);
                double ey = d->x[2 * k + 1] - yj;
                double Rk = ri + d->r[k];
                double e2 = ex * ex + ey * ey;
                double e = sqrt(e2);
                if (e >= R + Rk || e <= fabs(R - Rk)) continue;
                /* points on the circle |p| = R (around j) with |p - e| = Rk:
                 * p . e = (R^2 + e^2 - Rk^2) / 2 */
                double proj = (R * R + e2 - Rk * Rk) / (2.0 * e);
                double h2 = R * R - proj * proj;
                if (h2 < 0.0) continue;
                double h = sqrt(h2);
                double ux = ex / e, uy = ey / e;
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    double px = proj * ux + sgn * h * (-uy);
                    double py = proj * uy + sgn * h * ux;
                    /* angle from vertical on side s: px = s R sin(phi), py = R cos(phi) */
                    if (s * px < -1e-12) continue;
                    double phi = atan2(s * px, py);
                    if (phi > phi0 + 1e-12 && phi < best) { best = phi; who = k; }
                }
            }
        }
    }
    *phi_out = best;
    return who;
}

static void depo_insert(depo* d, int64_t i)
{
    int64_t c = col_of(d, d->x[2 * i]);
    int64_t row = row_of(d, d->x[2 * i + 1]);
    int64_t cell = row * d->ncx + c;
    d->next[i] = d->head[cell];
    d->head[cell] = i;
    if (row > d->coltop[c]) d->coltop[c] = row;
}

/* Returns the number of discs deposited (n unless the height limit is hit). */
int64_t wl_deposit2d(int64_t n, const double* radii, double Lx, double ymax, uint64_t seed, double* x)
{
    depo d;
    d.r = radii;
    d.x = x;
    d.Lx = Lx;
    d.rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (radii[i] > d.rmax) d.rmax = radii[i];
    d.ncx = (int64_t)floor(Lx / (2.0 * d.rmax));
    if (d.ncx < 3) d.ncx = 3;
    d.cs = Lx / (double)d.ncx;
    d.ncy = (int64_t)ceil(ymax / d.cs) + 4;
    d.head = (int64_t*)malloc(sizeof(int64_t) * (size_t)(d.ncx * d.ncy));
    d.next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    d.coltop = (int64_t*)malloc(sizeof(int64_t) * (size_t)d.ncx);
    for (int64_t c = 0; c < d.ncx * d.ncy; ++c) d.head[c] = -1;
    for (int64_t c = 0; c < d.ncx; ++c) d.coltop[c] = -1;
    uint64_t s = seed;
    int64_t placed = 0;
    for (int64_t i = 0; i < n; ++i) {
        double ri = radii[i];
        double xi = Lx * u01(&s);
        double yi;
        int64_t sup = fall(&d, xi, ri, 1e300, -1, &yi);
        int iter = 0;
        while (sup >= 0 && iter < 400) {
            ++iter;
            double xj = d.x[2 * sup], yj = d.x[2 * sup + 1];
            double R = ri + radii[sup];
            double dx = min_image(xi - xj, Lx, 1);
            int sd = (dx > 0.0) ? 1 : (dx < 0.0 ? -1 : ((sm64_next(&s) & 1) ? 1 : -1));
            double phi0 = atan2(fabs(dx), yi - yj);
            double phi;
            int64_t k = roll(&d, ri, sup, phi0, sd, &phi);
            double nx = xj + sd * R * sin(phi), ny = yj + R * cos(phi);
            nx = fmod(nx, Lx);
            if (nx < 0.0) nx += Lx;
            xi = nx; yi = ny;
            if (k == -1) { sup = -1; break; }             /* rests on the floor */
            if (k == -2) {                                /* rolled off: fall again */
                sup = fall(&d, xi, ri, yi, sup, &yi);
                continue;
            }
            double dk = min_image(d.x[2 * k] - xi, Lx, 1);
            double dj = min_image(xj - xi, Lx, 1);
            if ((dk > 0.0) != (dj > 0.0)) break;          /* supports on both sides: stable */
            sup = k;                                      /* roll on over the new support */
        }
        if (yi + ri > ymax) break;
        x[2 * i] = xi;
        x[2 * i + 1] = yi;
        depo_insert(&d, i);
        ++placed;
    }
    free(d.coltop); free(d.next); free(d.head);
    return placed;
}
