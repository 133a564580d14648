// Domain-wise update of the parallel algorithm (Sec. 3.1) on one GPU: the
// per-step setup of the domain views.
//
// In the paper every processor sweeps the contacts of its domain
// sequentially while the contacts of its neighbours (foreign contacts) keep
// the forces of the previous sweep; the new forces are exchanged at the end
// of the sweep.  On one GPU a domain's view of a particle is a velocity
// record of its own: a particle whose contacts lie in several domains gets
// one record per domain (its own record for the lowest domain, view records
// after the walls' records for the others).  The sweep kernel updates every
// contact on its domain's records, and after each sweep adds the records'
// changes into the particle's velocity and copies the sum back into every
// view (cd_sweep.cu).  This file assigns contacts to domains and builds the
// record map.
#include "cd_internal.cuh"

// Domain of key-order contact c: the slab grid over the box, by the middle of
// the gap q = x_a + n (r_a + g / 2), wrapped once on a periodic axis; slab
// floor(((q - lo) / (hi - lo)) * nd), clamped; id = ix + nx (iy + ny iz).
// Every operation is rounded as written (no contraction).
__device__ __forceinline__ int contact_domain(const CdGeom& g, const CdWork& w, const double* __restrict__ pos,
                                              const double* __restrict__ radius, int c)
{
    const int a = w.pairs[c].x;
    const double half = __dadd_rn(radius[a], __dmul_rn(0.5, w.gap[c]));
    int id = 0, mult = 1;
    for (int k = 0; k < g.dim; ++k) {
        const int nd = g.ndom[k];
        if (nd > 1) {
            const double lo = g.lo[k], hi = g.hi[k];
            double q = __dadd_rn(pos[(size_t)a * g.dim + k], __dmul_rn(w.nrm[3 * c + k], half));
            if (g.periodic[k]) {
                if (q >= hi) q = __dsub_rn(q, __dsub_rn(hi, lo));
                else if (q < lo) q = __dadd_rn(q, __dsub_rn(hi, lo));
            }
            const double t = __dmul_rn(__ddiv_rn(__dsub_rn(q, lo), __dsub_rn(hi, lo)), (double)nd);
            long long ix = (long long)floor(t);
            if (ix < 0) ix = 0;
            if (ix > nd - 1) ix = nd - 1;
            id += (int)ix * mult;
        }
        mult *= nd;
    }
    return id;
}

__global__ void k_dom_contact(CdGeom g, CdWork w, const double* __restrict__ pos, const double* __restrict__ radius)
{
    if (w.ctrl->skip) return;
    const int nc = w.ctrl->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
        w.dom_key[c] = contact_domain(g, w, pos, radius, c);
}

// True if the s-th entry of particle i's contact list is the first one with
// its domain.
__device__ __forceinline__ bool first_of_domain(const CdWork& w, int b, int s, int d)
{
    for (int u = b; u < s; ++u)
        if (w.dom_key[w.p2c[u]] == d) return false;
    return true;
}

// Distinct domains of particle i below d (its list is short: its contacts).
__device__ __forceinline__ int domains_below(const CdWork& w, int i, int d)
{
    const int b = w.p2c_off[i], e = w.p2c_off[i + 1];
    int cnt = 0;
    for (int s = b; s < e; ++s) {
        const int x = w.dom_key[w.p2c[s]];
        if (x < d && first_of_domain(w, b, s, x)) ++cnt;
    }
    return cnt;
}

// Home domain and number of view records of every particle.
__global__ void k_dom_count(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        const int b = w.p2c_off[i], e = w.p2c_off[i + 1];
        int home = -1, distinct = 0;
        for (int s = b; s < e; ++s) {
            const int d = w.dom_key[w.p2c[s]];
            if (home < 0 || d < home) home = d;
            if (first_of_domain(w, b, s, d)) ++distinct;
        }
        w.dom_home[i] = home;
        w.view_cnt[i] = distinct > 1 ? distinct - 1 : 0;
    }
}

// Owner of every view record: view_off[i] + (rank of the domain among i's
// domains) - 1.
__global__ void k_dom_owner(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        if (w.view_cnt[i] == 0) continue;
        const int b = w.p2c_off[i], e = w.p2c_off[i + 1], home = w.dom_home[i];
        for (int s = b; s < e; ++s) {
            const int d = w.dom_key[w.p2c[s]];
            if (d == home || !first_of_domain(w, b, s, d)) continue;
            w.view_owner[w.view_off[i] + domains_below(w, i, d) - 1] = i;
        }
    }
}

__device__ __forceinline__ int view_record(const CdGeom& g, const CdWork& w, int i, int d)
{
    if (d == w.dom_home[i]) return i;
    return cd_view_base(g) + w.view_off[i] + domains_below(w, i, d) - 1;
}

// Velocity records of the two bodies of every colour-order contact.
__global__ void k_dom_vab(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    const int nc = w.ctrl->nc;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nc; p += gridDim.x * blockDim.x) {
        const int2 ab = w.c_ab[p];
        const int d = w.dom_key[w.perm[p]];
        int2 v;
        v.x = view_record(g, w, ab.x, d);
        v.y = (ab.y < g.n) ? view_record(g, w, ab.y, d) : ab.y;   // kinematic walls keep their id
        w.c_vab[p] = v;
    }
}

cudaError_t cd_launch_domains(const CdGeom& g, const CdWork& w, const double* pos, const double* radius,
                              cudaStream_t s, int* nl)
{
    cudaError_t e;
    int gc = (g.cap + CD_BLOCK - 1) / CD_BLOCK;
    if (gc < 1) gc = 1;
    if (gc > 4096) gc = 4096;
    int gn = (g.n + CD_BLOCK - 1) / CD_BLOCK;
    if (gn < 1) gn = 1;
    if (gn > 4096) gn = 4096;
    k_dom_contact<<<gc, CD_BLOCK, 0, s>>>(g, w, pos, radius); ++*nl;
    if ((e = cudaMemsetAsync(w.view_cnt, 0, sizeof(int) * (size_t)(g.n + 1), s)) != cudaSuccess) return e;
    k_dom_count<<<gn, CD_BLOCK, 0, s>>>(g, w); ++*nl;
    if ((e = cd_scan_exclusive(w.view_cnt, w.view_off, g.n + 1, w.scan_tmp, nullptr, s, nl)) != cudaSuccess)
        return e;
    k_dom_owner<<<gn, CD_BLOCK, 0, s>>>(g, w); ++*nl;
    k_dom_vab<<<gc, CD_BLOCK, 0, s>>>(g, w); ++*nl;
    return cudaGetLastError();
}
