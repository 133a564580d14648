// cd_detect.cu -- contact detection with a cell list (paper Sec. 3.2) and the
// per-contact geometry (Sec. 2.1, Fig. 1; pair mass matrix of Eq. 5).
//
// Pipeline (all on one stream, sizes read from the control block so nothing
// is synchronised with the host):
//   cell_count -> scan -> cell_fill, sort    counting sort of particles by cell
//   pair_count -> scan -> capacity check     contacts per particle a (b > a)
//   pair_emit                                keys (a, b) sorted per a
//   geometry_warm -> commit                  geometry per contact, impulses carried over by key
// The pair test uses the same FP64 operation sequence as the CPU oracle
// (explicit round-to-nearest intrinsics, no FMA contraction) so the contact
// set is bit-identical to brute force.
#include <climits>

#include "cd_internal.cuh"

// ---------------------------------------------------------------------------
// Exclusive scan of int32: the block sums of the tiles, then every block
// scans its tile and adds the prefix of the tiles before it.  Up to
// SCAN_FUSE tiles each block sums that prefix itself from the block sums
// (read by all blocks from L2; integer sums, so the order is immaterial);
// beyond, a single block scans the block sums in between (three passes).
// `n_dev` (device, optional) clips the scan at run time to its first
// min(*n_dev + 1, n) entries (the rest of `out` is left untouched), for
// arrays sized by capacity of which only the live contacts count.
// `total_dst` (device) receives the sum of the scanned inputs if non-null.
// In place (in == out) is allowed: a tile is read and written by the same
// threads.
// ---------------------------------------------------------------------------
#define SCAN_T 256
#define SCAN_PER 4
#define SCAN_TILE (SCAN_T * SCAN_PER)
#define SCAN_FUSE 2048

__device__ __forceinline__ int scan_extent(int n, const int* n_dev)
{
    if (!n_dev) return n;
    const int c = *n_dev + 1;
    return (c < n) ? c : n;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ int block_excl_scan(int v, int* total)
{
    __shared__ int warp_sums[SCAN_T / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < SCAN_T / 32) ? warp_sums[lane] : 0;
        int si = warp_incl_scan(s);
        if (lane < SCAN_T / 32) warp_sums[lane] = si - s;
        if (lane == SCAN_T / 32 - 1) *total = si;
    }
    __syncthreads();
    int r = warp_sums[wid] + incl - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_sums(const int* __restrict__ in, int n, const int* n_dev, int* __restrict__ sums)
{
    n = scan_extent(n, n_dev);
    int base = blockIdx.x * SCAN_TILE;
    if (base >= n) return;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        int i = base + k * SCAN_T + threadIdx.x;
        if (i < n) s += in[i];
    }
    __shared__ int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Three-pass form only: one block turns the block sums into their exclusive
// prefixes.
__global__ void k_scan_top(int* sums, int n, const int* n_dev, int* total_dst)
{
    n = scan_extent(n, n_dev);
    const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += SCAN_T) {
        int i = base + threadIdx.x;
        int v = (i < nb) ? sums[i] : 0;
        __shared__ int tot;
        int ex = block_excl_scan(v, &tot);
        int carry = carry_s;
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total_dst) *total_dst = carry_s;
}

// fused: the prefix of this tile from the raw block sums (else sums already
// holds the prefixes)
__global__ void k_scan_apply(const int* in, int n, const int* n_dev, const int* __restrict__ sums, int fused,
                             int* out, int* total_dst)
{
    n = scan_extent(n, n_dev);
    const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if ((int)blockIdx.x >= nb) return;
    __shared__ int prefix;
    if (fused) {
        int p = 0;
        for (int j = threadIdx.x; j < (int)blockIdx.x; j += SCAN_T) p += sums[j];
        block_excl_scan(p, &prefix);
    } else {
        if (threadIdx.x == 0) prefix = sums[blockIdx.x];
        __syncthreads();
    }
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
    int v[SCAN_PER];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        int i = base + k;
        v[k] = (i < n) ? in[i] : 0;
        s += v[k];
    }
    __shared__ int tot;
    int ex = block_excl_scan(s, &tot) + prefix;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        int i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
    if (fused && total_dst && (int)blockIdx.x == nb - 1 && threadIdx.x == 0) *total_dst = prefix + tot;
}

size_t cd_scan_tmp_ints(int n)
{
    return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE + 1);
}

cudaError_t cd_scan_exclusive(const int* in, int* out, int n, int* tmp, int* total_dst, cudaStream_t stream,
                              int* nl, const int* n_dev)
{
    if (n <= 0) return cudaSuccess;
    int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    const int fused = (nb <= SCAN_FUSE || n_dev) ? 1 : 0;
    k_scan_sums<<<nb, SCAN_T, 0, stream>>>(in, n, n_dev, tmp);
    if (!fused) {
        k_scan_top<<<1, SCAN_T, 0, stream>>>(tmp, n, n_dev, total_dst);
        ++*nl;
    }
    k_scan_apply<<<nb, SCAN_T, 0, stream>>>(in, n, n_dev, tmp, fused, out, total_dst);
    *nl += 2;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cell list.  Every packing of a batched system has its own grid (a plain
// system is one packing); global cell id = the packing's cell_base + local id,
// so particles of different packings are never in neighbouring cells.
// ---------------------------------------------------------------------------
struct GridV {
    double lo[3], cs[3], inv_cs[3], L[3];
    int ncell[3], periodic[3];
    int base, wall_mask, pkid;
};

__device__ __forceinline__ void grid_of(const CdGeom& g, const CdWork& w, int i, GridV& v)
{
    if (g.npk > 1) {
        const int b = w.pack_of[i];
        const CdPack& p = w.pk[b];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            v.lo[k] = p.lo[k]; v.cs[k] = p.cs[k]; v.inv_cs[k] = p.inv_cs[k]; v.L[k] = p.L[k];
            v.ncell[k] = p.ncell[k]; v.periodic[k] = p.periodic[k];
        }
        v.base = p.cell_base; v.wall_mask = p.wall_mask; v.pkid = b;
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            v.lo[k] = g.lo[k]; v.cs[k] = g.cs[k]; v.inv_cs[k] = g.inv_cs[k]; v.L[k] = g.L[k];
            v.ncell[k] = g.ncell[k]; v.periodic[k] = g.periodic[k];
        }
        v.base = 0; v.wall_mask = g.wall_mask; v.pkid = 0;
    }
}

// Cell index along axis k: floor((x - lo) / cs) clamped to the grid, with
// the quotient taken as a product by 1 / cs and rounded down to an integer
// in one conversion (a correctly rounded FP64 division is ~10 FP64
// instructions).  Either rounding may put a particle within a few ulps of a
// cell face into the neighbouring cell; no contact is lost: a contact is
// closer than r_a + r_b + delta <= 2 r_max + delta, the cell side is longer
// than that by a relative 1e-9 (far more than the misplacement, on grids of
// up to 1e6 cells per axis), and the pair walk visits every cell next to the
// one a particle is filed in.  (A NaN coordinate converts to 0: cell 0.)
__device__ __forceinline__ int cell_axis(const GridV& v, int k, double x)
{
    const int q = __double2int_rd(__dmul_rn(__dsub_rn(x, v.lo[k]), v.inv_cs[k]));
    return q < 0 ? 0 : (q > v.ncell[k] - 1 ? v.ncell[k] - 1 : q);
}

template <int DIM>
__global__ void k_cell_count(CdGeom g, CdWork w, const double* __restrict__ pos, const double* __restrict__ radius,
                             int* __restrict__ cell_of, int* __restrict__ cell_cnt, const CdCtrl* ctrl)
{
    if (ctrl->skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        GridV v;
        grid_of(g, w, i, v);
        if (w.pf) {
            // single-precision copy of (x, y, z, r) for the pair pre-filter
            w.pf[i] = make_float4((float)pos[i * DIM + 0], (float)pos[i * DIM + 1],
                                  DIM == 3 ? (float)pos[i * DIM + 2] : 0.0f, (float)radius[i]);
        }
        int c0 = cell_axis(v, 0, pos[i * DIM + 0]);
        int c1 = cell_axis(v, 1, pos[i * DIM + 1]);
        int c2 = (DIM == 3) ? cell_axis(v, 2, pos[i * DIM + 2]) : 0;
        int c = v.base + (c2 * v.ncell[1] + c1) * v.ncell[0] + c0;
        cell_of[i] = c;
        atomicAdd(&cell_cnt[c], 1);
    }
}

__global__ void k_cell_fill(int n, const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                            int* __restrict__ cell_fill, int* __restrict__ cell_pid, const CdCtrl* ctrl)
{
    if (ctrl->skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c = cell_of[i];
        int slot = atomicAdd(&cell_fill[c], 1);
        cell_pid[cell_start[c] + slot] = i;
    }
}

// Each cell's particle list in ascending id order (the atomic fill leaves it
// in arrival order): lets the pair walk skip a whole cell whose last id is
// not above the particle's own.
__global__ void k_cell_sort(int ncell, const int* __restrict__ cell_start, int* __restrict__ cell_pid,
                            const CdCtrl* ctrl)
{
    if (ctrl->skip) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const int b = cell_start[c], e = cell_start[c + 1];
        for (int k = b + 1; k < e; ++k) {
            const int v = cell_pid[k];
            int j = k - 1;
            while (j >= b && cell_pid[j] > v) { cell_pid[j + 1] = cell_pid[j]; --j; }
            cell_pid[j + 1] = v;
        }
    }
}

// Separation b - a along axis k with the minimum-image rule (same operations
// as the oracle).
__device__ __forceinline__ double sep_axis(const GridV& v, int k, double xa, double xb)
{
    double d = __dsub_rn(xb, xa);
    if (v.periodic[k]) {
        double half = __dmul_rn(0.5, v.L[k]);
        if (d > half) d = __dsub_rn(d, v.L[k]);
        else if (d < -half) d = __dadd_rn(d, v.L[k]);
    }
    return d;
}

template <int DIM>
__device__ __forceinline__ bool pair_touches(const GridV& v, double delta, const double* xa, double ra,
                                             const double* __restrict__ pos, const double* __restrict__ radius, int b)
{
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double d = sep_axis(v, k, xa[k], pos[b * DIM + k]);
        double dd = __dmul_rn(d, d);
        d2 = (k == 0) ? dd : __dadd_rn(d2, dd);
    }
    double s = __dadd_rn(__dadd_rn(ra, radius[b]), delta);
    return d2 < __dmul_rn(s, s);
}

// Single-precision pre-filter of the pair test: true only if the pair is
// certainly not a contact, so that the exact FP64 test above (which alone
// decides) runs only for the candidates that may be.  Each coordinate
// rounded to float is within 2^-24 |x| of the double, so the float
// separation of an axis is within e_k = 2^-23 (|x_a| + |x_b| (+ L on a
// periodic axis)) of the exact one (a factor two over the rounding of the
// conversions, the subtraction and the image shift), and the distance
// within E = sum_k e_k.  A contact has |d| < s, hence a float distance
// below s + E; the relative roundings of d2, of s and of the threshold
// itself are covered by the factors 1 + 2^-20.  An image chosen differently
// near |d| = L/2 changes nothing: a periodic axis spans at least three cells,
// so both images are farther apart than any contact distance.
template <int DIM>
__device__ __forceinline__ bool pair_far_f32(const GridV& v, const float (&Lf)[3], float delta_f, const float4& pa,
                                             const float4& pb)
{
    const float xa[3] = {pa.x, pa.y, pa.z}, xb[3] = {pb.x, pb.y, pb.z};
    float d2 = 0.0f, E = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        float d = xb[k] - xa[k];
        float m = fabsf(xa[k]) + fabsf(xb[k]);
        if (v.periodic[k]) {
            const float half = 0.5f * Lf[k];
            if (d > half) d -= Lf[k];
            else if (d < -half) d += Lf[k];
            m += Lf[k];
        }
        d2 = fmaf(d, d, d2);
        E = fmaf(m, 1.1920929e-7f, E);   // 2^-23
    }
    const float s = pa.w + pb.w + delta_f;
    const float t = fmaf(s, 1.0f + 9.5367432e-7f, E) * (1.0f + 9.5367432e-7f);   // 1 + 2^-20
    return d2 > t * t;
}

// Gap of the particle at xa to wall k (k = 2 axis + side).  The coordinate is
// picked by selects, not by indexing xa with k (a run-time index would put
// the caller's small arrays in local memory).
__device__ __forceinline__ double wall_gap(const double* xa, double ra, const double* wall_pos, int k)
{
    const int axis = k >> 1;
    const double x = (axis == 0) ? xa[0] : (axis == 1) ? xa[1] : xa[2];
    if ((k & 1) == 0) return __dsub_rn(__dsub_rn(x, wall_pos[k]), ra);
    return __dsub_rn(__dsub_rn(wall_pos[k], x), ra);
}

__device__ __forceinline__ bool wall_on(const GridV& v, int dim, int k)
{
    return ((v.wall_mask >> k) & 1) && (k >> 1) < dim;
}

// Walls in contact with the particle at xa (bit k: wall k has gap < delta).
template <int DIM>
__device__ __forceinline__ unsigned wall_mask_of(const CdGeom& g, const GridV& v, const double* wp, const double* xa,
                                                 double ra)
{
    unsigned m = 0u;
#pragma unroll
    for (int k = 0; k < 2 * DIM; ++k)
        if (wall_on(v, DIM, k) && wall_gap(xa, ra, wp, k) < g.delta) m |= 1u << k;
    return m;
}

// Visits the candidate partners b > a of particle a in the 3^DIM cells around
// it (in a's packing grid); calls f(b) for each b that passes the pair test.
// Needs each cell's list sorted by id (k_cell_sort).
//
// The three cells x-1, x, x+1 of one row of the stencil are consecutive cell
// ids, so their particles are one run of cell_pid: 3^(DIM-1) runs (a periodic
// x axis that wraps adds the wrapped cell as a run of its own).  A cell whose
// last id is not above a holds no partner: such cells are trimmed off the
// left end of a run, and a run none of whose cells passes is dropped (ids
// follow the packing's rows, so that is most runs below a's row).  The
// candidates of the runs are then walked as one flat sequence, so the lanes
// of a warp loop about as many times as their own candidate counts.  The
// runs' bounds live in registers (RUNS fixed, the loops unrolled, the next
// run picked by comparisons against compile-time indices): an array of cell
// ranges indexed in a loop went to local memory and dominated the kernel's
// memory traffic.
template <int DIM>
struct Runs {
    static constexpr int N = (DIM == 3) ? 18 : 6;   // 3^(DIM-1) rows, each with a possible wrapped cell
    int lo[N], hi[N];
    // r is a compile-time index at every call (unrolled loops)
    __device__ __forceinline__ void set(int r, int l, int h) { lo[r] = l; hi[r] = h; }
    __device__ __forceinline__ void get(int j, int& l, int& h) const
    {
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k == j) { l = lo[k]; h = hi[k]; }
    }
};

// The same runs in shared memory, [run][thread] (a warp's accesses fall in
// distinct banks): the counting pass keeps its registers for the walk
// itself, and a run is fetched by its run-time index.
template <int DIM>
struct RunsShared {
    static constexpr int N = Runs<DIM>::N;
    int* lo;   // &s_lo[0][threadIdx.x], stride CD_BLOCK
    int* hi;
    __device__ __forceinline__ void set(int r, int l, int h) { lo[r * CD_BLOCK] = l; hi[r * CD_BLOCK] = h; }
    __device__ __forceinline__ void get(int j, int& l, int& h) const { l = lo[j * CD_BLOCK]; h = hi[j * CD_BLOCK]; }
};

__device__ __forceinline__ int last_id(const int* __restrict__ cell_start, const int* __restrict__ cell_pid, int cc)
{
    const int l = cell_start[cc], h = cell_start[cc + 1];
    return (h > l) ? cell_pid[h - 1] : -1;
}

// Builds the runs of particle a in R (Runs or RunsShared); the walk starts
// at run 0.
template <int DIM, typename RS>
__device__ __forceinline__ void walk_init(const GridV& v, int a, const int* __restrict__ cell_of,
                                          const int* __restrict__ cell_start, const int* __restrict__ cell_pid,
                                          RS& R)
{
    const int c = cell_of[a] - v.base;
    const int n0 = v.ncell[0], n1 = v.ncell[1];
    const int q0 = c % n0;
    const int q1 = (c / n0) % n1;
    const int q2 = c / (n0 * n1);
    const int x0 = (q0 > 0) ? q0 - 1 : 0, x1 = (q0 < n0 - 1) ? q0 + 1 : n0 - 1;
    int xw = -1;   // a periodic x axis: the wrapped neighbour cell outside [x0, x1]
    if (v.periodic[0] && n0 >= 3) {
        if (q0 == 0) xw = n0 - 1;
        else if (q0 == n0 - 1) xw = 0;
    }
    constexpr int ZN = (DIM == 3) ? 3 : 1;
#pragma unroll
    for (int iz = 0; iz < ZN; ++iz) {
#pragma unroll
        for (int iy = 0; iy < 3; ++iy) {
            const int r = 2 * (iz * 3 + iy);
            int l0 = 0, h0 = 0, l1 = 0, h1 = 0;
            int t2 = (DIM == 3) ? q2 + iz - 1 : 0;
            if (DIM == 3 && (t2 < 0 || t2 >= v.ncell[2])) {
                if (!v.periodic[2]) { R.set(r, 0, 0); R.set(r + 1, 0, 0); continue; }
                t2 = (t2 + v.ncell[2]) % v.ncell[2];
            }
            int t1 = q1 + iy - 1;
            if (t1 < 0 || t1 >= n1) {
                if (!v.periodic[1]) { R.set(r, 0, 0); R.set(r + 1, 0, 0); continue; }
                t1 = (t1 + n1) % n1;
            }
            const int row = v.base + (t2 * n1 + t1) * n0;
            // the run's cells x0 .. x1 (one to three): their bounds, then their last
            // ids (independent loads); the run starts at its first cell with an id above a
            const int nx = x1 - x0 + 1;
            const int cs0 = cell_start[row + x0];
            const int cs1 = (nx > 1) ? cell_start[row + x0 + 1] : 0;
            const int cs2 = (nx > 2) ? cell_start[row + x0 + 2] : 0;
            const int cs3 = cell_start[row + x1 + 1];
            const int e0 = (nx > 1) ? cs1 : cs3, e1 = (nx > 2) ? cs2 : cs3;
            const int L0 = (e0 > cs0) ? cell_pid[e0 - 1] : -1;
            const int L1 = (nx > 1 && e1 > cs1) ? cell_pid[e1 - 1] : -1;
            const int L2 = (nx > 2 && cs3 > cs2) ? cell_pid[cs3 - 1] : -1;
            const int start = (L0 > a) ? cs0 : (L1 > a) ? cs1 : (L2 > a) ? cs2 : -1;
            if (start >= 0) {
                l0 = start;
                h0 = cs3;
            }
            if (xw >= 0 && last_id(cell_start, cell_pid, row + xw) > a) {
                l1 = cell_start[row + xw];
                h1 = cell_start[row + xw + 1];
            }
            R.set(r, l0, h0);
            R.set(r + 1, l1, h1);
        }
    }
}

// The next candidate of the flat walk over the runs (j the run, [s, e) what
// is left of it), or -1 once they are exhausted (and on every later call).
template <int DIM, typename RS>
__device__ __forceinline__ int walk_next(const RS& R, int& j, int& s, int& e, const int* __restrict__ cell_pid)
{
    while (s >= e) {
        if (++j >= Runs<DIM>::N) return -1;
        R.get(j, s, e);
    }
    return cell_pid[s++];
}

template <int DIM, typename F>
__device__ __forceinline__ void for_each_partner(const CdGeom& g, const GridV& v, int a, const double* xa, double ra,
                                                 const double* __restrict__ pos, const double* __restrict__ radius,
                                                 const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                                                 const int* __restrict__ cell_pid, const float4* __restrict__ pf, F f)
{
    Runs<DIM> R;
    walk_init<DIM>(v, a, cell_of, cell_start, cell_pid, R);
    int j = 0, s = R.lo[0], e = R.hi[0];
    // the pre-filter's data (pf null: the exact test only)
    float4 pa = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float Lf[3] = {(float)v.L[0], (float)v.L[1], (float)v.L[2]};
    const float delta_f = (float)g.delta;
    if (pf) pa = pf[a];
    for (;;) {
        const int b = walk_next<DIM>(R, j, s, e, cell_pid);
        if (b < 0) break;
        if (b > a && !(pf && pair_far_f32<DIM>(v, Lf, delta_f, pa, pf[b])) &&
            pair_touches<DIM>(v, g.delta, xa, ra, pos, radius, b))
            f(b);
    }
}

// Exact tests of the first `take` queued pairs of a warp, lane q on pair q:
// the owner lane's particle (its id, position and radius by shuffles), the
// partner's from memory.  A pair that touches counts for its owner and is
// kept among the owner's first CD_CAND partners.
template <int DIM>
__device__ __forceinline__ void exact_batch(const CdGeom& g, const CdWork& w, const double* __restrict__ pos,
                                            const double* __restrict__ radius, int a, double x0, double x1,
                                            double x2, double ra, int take, const int* qb, const int* qo, int* cnt)
{
    const int lane = threadIdx.x & 31;
    const int o = (lane < take) ? qo[lane] : 0;
    const int b = (lane < take) ? qb[lane] : 0;
    const int ao = __shfl_sync(0xffffffffu, a, o);
    double xo[3];
    xo[0] = __shfl_sync(0xffffffffu, x0, o);
    xo[1] = __shfl_sync(0xffffffffu, x1, o);
    xo[2] = (DIM == 3) ? __shfl_sync(0xffffffffu, x2, o) : 0.0;
    const double ro = __shfl_sync(0xffffffffu, ra, o);
    if (lane < take) {
        GridV vo;
        grid_of(g, w, ao, vo);
        if (pair_touches<DIM>(vo, g.delta, xo, ro, pos, radius, b)) {
            const int slot = atomicAdd(&cnt[o], 1);
            if (w.cand && slot < CD_CAND) w.cand[(size_t)ao * CD_CAND + slot] = b;
        }
    }
}

// Counting pass: partners b > a of every particle, and its walls.  A lane
// walks its particle's candidates through the single-precision pre-filter;
// the candidates that pass are queued per warp (ballot and prefix count) and
// the warp runs the exact FP64 test on 32 queued pairs at a time, whoever
// owns them.  With the test inside the walk the warp issued it in nearly
// every step, since some lane's candidate nearly always passes the
// pre-filter (~220 FP64 warp instructions per particle warp on the
// 1e6-sphere gas).  The partners found and their count are those of the
// walk; only the order in which a particle's first CD_CAND partners are kept
// depends on timing, and the emitting pass sorts them.  The runs live in
// shared memory and the walk's state in registers: 64 registers, four
// blocks per SM without spills.  The particle's wall contacts are kept as a
// bit mask for the emitting pass.
template <int DIM>
__global__ void __launch_bounds__(CD_BLOCK, 4)
k_pair_count(CdGeom g, CdWork w, const double* __restrict__ pos, const double* __restrict__ radius,
                             const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                             const int* __restrict__ cell_pid, int* __restrict__ pcnt, CdCtrl* ctrl)
{
    __shared__ int s_qb[CD_BLOCK / 32][64];   // queued partners (at most 31 left over + 32 new)
    __shared__ int s_qo[CD_BLOCK / 32][64];   // their owner lanes
    __shared__ int s_cnt[CD_BLOCK];
    __shared__ int s_lo[Runs<DIM>::N][CD_BLOCK], s_hi[Runs<DIM>::N][CD_BLOCK];
    if (ctrl->skip) return;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    int* const qb = s_qb[wq];
    int* const qo = s_qo[wq];
    int* const cnt_w = s_cnt + 32 * wq;
    // warps step through the particles together (the loop bound is warp-uniform)
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < g.n; base += gridDim.x * blockDim.x) {
        const int a = base + lane;
        const bool act = a < g.n;
        GridV v;
        double xa[3] = {0.0, 0.0, 0.0};
        double ra = 0.0;
        RunsShared<DIM> R;
        R.lo = &s_lo[0][threadIdx.x];
        R.hi = &s_hi[0][threadIdx.x];
        int j = 0, s = 0, e = 0;
        float4 pa = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float Lf[3] = {0.0f, 0.0f, 0.0f};
        bool more = act;
        if (act) {
            grid_of(g, w, a, v);
#pragma unroll
            for (int k = 0; k < DIM; ++k) xa[k] = pos[a * DIM + k];
            ra = radius[a];
            walk_init<DIM>(v, a, cell_of, cell_start, cell_pid, R);
            R.get(0, s, e);
            if (w.pf) pa = w.pf[a];
#pragma unroll
            for (int k = 0; k < 3; ++k) Lf[k] = (float)v.L[k];
        }
        const float delta_f = (float)g.delta;
        s_cnt[threadIdx.x] = 0;
        __syncwarp();
        int qn = 0;   // queued pairs (the same in every lane)
        for (;;) {
            int b = -1;
            bool q = false;
            if (more) {
                b = walk_next<DIM>(R, j, s, e, cell_pid);
                if (b < 0) more = false;
                else q = b > a && !(w.pf && pair_far_f32<DIM>(v, Lf, delta_f, pa, w.pf[b]));
            }
            const unsigned m = __ballot_sync(0xffffffffu, q);
            if (q) {
                const int at = qn + __popc(m & ((1u << lane) - 1u));
                qb[at] = b;
                qo[at] = lane;
            }
            qn += __popc(m);
            const bool done = !__any_sync(0xffffffffu, more);
            while (qn >= 32 || (done && qn > 0)) {
                __syncwarp();
                const int take = qn < 32 ? qn : 32;
                exact_batch<DIM>(g, w, pos, radius, a, xa[0], xa[1], xa[2], ra, take, qb, qo, cnt_w);
                // the rest (fewer than 32) to the front of the queue
                const int rest = qn - take;
                int rb = 0, ro = 0;
                if (lane < rest) { rb = qb[32 + lane]; ro = qo[32 + lane]; }
                __syncwarp();
                if (lane < rest) { qb[lane] = rb; qo[lane] = ro; }
                __syncwarp();
                qn = rest;
            }
            if (done) break;
        }
        __syncwarp();
        if (act) {
            const int cnt = s_cnt[threadIdx.x];
            const unsigned wm = wall_mask_of<DIM>(g, v, w.pk_wall_pos + 6 * v.pkid, xa, ra);
            if (w.wmask) w.wmask[a] = (unsigned char)wm;   // the emitting pass reuses it
            if (cnt > CD_MAXLOC) atomicCAS(&ctrl->error, CDE_NONE, CDE_PER_PARTICLE);
            pcnt[a] = cnt + __popc(wm);
        }
        __syncwarp();
    }
}

// Capacity check after the scan of the per-particle counts.
__global__ void k_cap_check(CdCtrl* ctrl, int cap)
{
    if (ctrl->skip) return;
    if (ctrl->nc_needed > cap || ctrl->error != CDE_NONE) {
        ctrl->overflow = (ctrl->nc_needed > cap) ? 1 : ctrl->overflow;
        ctrl->skip = 1;
    }
}

// Geometry of contact (a, b): normal from a to b, gap, m_n = 1/w_n and
// m_t = 1/w_t with w_n = 1/m_a + 1/m_b, w_t = w_n + r_a^2/I_a + r_b^2/I_b.
// A wall is body n + 6 * packing + k.
template <int DIM>
__device__ __forceinline__ void contact_geometry(const CdGeom& g, const CdWork& w, int a, int b,
                                                 const double* __restrict__ pos, const double* __restrict__ radius,
                                                 const double* __restrict__ inv_m, const double* __restrict__ inv_I,
                                                 double nv[3], double* gap, double* mn, double* mt)
{
    GridV v;
    grid_of(g, w, a, v);
    double xa[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < DIM; ++k) xa[k] = pos[a * DIM + k];
    double ra = radius[a];
    double wa_m = inv_m[a], wa_I = g.rotations ? inv_I[a] : 0.0;
    double wb_m = 0.0, wb_I = 0.0, rb = 0.0;
    nv[0] = nv[1] = nv[2] = 0.0;
    if (b < g.n) {
        double dv[3] = {0.0, 0.0, 0.0};
        double d2 = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            dv[k] = sep_axis(v, k, xa[k], pos[b * DIM + k]);
            double dd = __dmul_rn(dv[k], dv[k]);
            d2 = (k == 0) ? dd : __dadd_rn(d2, dd);
        }
        double d = __dsqrt_rn(d2);
        if (d > 0.0) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) nv[k] = __ddiv_rn(dv[k], d);
        } else {
            nv[0] = 1.0;
        }
        rb = radius[b];
        *gap = __dsub_rn(d, __dadd_rn(ra, rb));
        wb_m = inv_m[b];
        wb_I = g.rotations ? inv_I[b] : 0.0;
    } else {
        int t = b - g.n;
        int k = t % 6;
        const double sgn = (k & 1) ? 1.0 : -1.0;
        const int axis = k >> 1;
        nv[0] = (axis == 0) ? sgn : 0.0;
        nv[1] = (axis == 1) ? sgn : 0.0;
        nv[2] = (axis == 2) ? sgn : 0.0;
        *gap = wall_gap(xa, ra, w.pk_wall_pos + 6 * (t / 6), k);
        // a force-controlled wall moves along its normal only: its inverse
        // mass enters the normal row, not the tangential one
        if (cd_is_body(g, b)) wb_m = g.wall_im[k];
    }
    double w_n = __dadd_rn(wa_m, wb_m);
    double w_t = __dadd_rn(__dadd_rn((b < g.n) ? w_n : wa_m, __dmul_rn(__dmul_rn(ra, ra), wa_I)),
                           __dmul_rn(__dmul_rn(rb, rb), wb_I));
    *mn = (w_n > 0.0) ? __ddiv_rn(1.0, w_n) : 0.0;
    *mt = (w_t > 0.0) ? __ddiv_rn(1.0, w_t) : 0.0;
}

template <int DIM>
__device__ __forceinline__ void store_geometry(const CdWork& w, int c, int a, int b, const double nv[3], double gap,
                                               double mn, double mt)
{
    w.pairs_nx[c] = make_int2(a, b);
    w.nrm[3 * c + 0] = nv[0];
    w.nrm[3 * c + 1] = nv[1];
    w.nrm[3 * c + 2] = nv[2];
    w.gap[c] = gap;
    w.mn[c] = mn;
    w.mt[c] = mt;
}

// Emitting pass: the keys (a, b) of every particle's contacts, partners in
// ascending id, then its walls, at the particle's offset from the scan of
// the counts.  Integer work only; the geometry follows one thread per
// contact (k_geometry_warm).
template <int DIM>
__global__ void k_pair_emit(CdGeom g, CdWork w, const double* __restrict__ pos, const double* __restrict__ radius)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.n; a += gridDim.x * blockDim.x) {
        GridV v;
        grid_of(g, w, a, v);
        double xa[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < DIM; ++k) xa[k] = pos[a * DIM + k];
        double ra = radius[a];
        // the counting pass's walls (the same test, so not repeated in FP64)
        const unsigned wm = w.wmask ? (unsigned)w.wmask[a]
                                    : wall_mask_of<DIM>(g, v, w.pk_wall_pos + 6 * v.pkid, xa, ra);
        const int npart = w.pcnt[a] - __popc(wm);   // partners the counting pass found
        int o = w.poff[a];
        if (w.cand && npart <= CD_CAND) {
            // the counting pass kept them (in the order its exact tests ran):
            // emit in ascending id by repeated selection of the smallest one
            // above the last emitted
            const int* keep = w.cand + (size_t)a * CD_CAND;
            int last = a;
            for (int f = 0; f < npart; ++f) {
                int bmin = INT_MAX;
                for (int q = 0; q < npart; ++q) {
                    const int bq = keep[q];
                    if (bq > last && bq < bmin) bmin = bq;
                }
                w.pairs_nx[o++] = make_int2(a, bmin);
                last = bmin;
            }
        } else {
            int found[CD_MAXLOC];
            int nf = 0;
            auto insert = [&](int b) {
                if (nf < CD_MAXLOC) {
                    // insertion into the sorted prefix
                    int j = nf++;
                    while (j > 0 && found[j - 1] > b) { found[j] = found[j - 1]; --j; }
                    found[j] = b;
                }
            };
            for_each_partner<DIM>(g, v, a, xa, ra, pos, radius, w.cell_of, w.cell_start, w.cell_pid, w.pf, insert);
            for (int f = 0; f < nf; ++f) w.pairs_nx[o++] = make_int2(a, found[f]);
        }
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k)
            if ((wm >> k) & 1u) w.pairs_nx[o++] = make_int2(a, g.n + 6 * v.pkid + k);
    }
}

// Geometry of every detected contact, one thread per contact (so that the
// FP64 square root and divisions run on full warps), and its starting
// impulse: matched by key in the current (previous) set; in 3D the old
// tangential impulse is projected onto the new tangent plane.
template <int DIM>
__global__ void k_geometry_warm(CdGeom g, CdWork w, const double* __restrict__ pos, const double* __restrict__ radius,
                                const double* __restrict__ inv_m, const double* __restrict__ inv_I, int warm, int pw)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    const int nnew = ctrl->nc_needed;
    const int nold = ctrl->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nnew; c += gridDim.x * blockDim.x) {
        const int2 ab = w.pairs_nx[c];
        double nv[3], gap, mn, mt;
        contact_geometry<DIM>(g, w, ab.x, ab.y, pos, radius, inv_m, inv_I, nv, &gap, &mn, &mt);
        w.nrm[3 * c + 0] = nv[0];
        w.nrm[3 * c + 1] = nv[1];
        w.nrm[3 * c + 2] = nv[2];
        w.gap[c] = gap;
        w.mn[c] = mn;
        w.mt[c] = mt;
        double out[4] = {0.0, 0.0, 0.0, 0.0};
        if (warm && nold > 0) {
            const unsigned long long key = cd_key(ab.x, ab.y);
            // the old set is in key order, so particle a's old contacts are the
            // range its offsets give (when kept), else somewhere in the whole set
            int lo = 0, hi = nold - 1, o = -1;
            if (ctrl->prev_offsets) {
                lo = w.poff_prev[ab.x];
                hi = w.poff_prev[ab.x + 1] - 1;
            }
            while (lo <= hi) {
                int mid = lo + ((hi - lo) >> 1);
                int2 m = w.pairs[mid];
                unsigned long long km = cd_key(m.x, m.y);
                if (km == key) { o = mid; break; }
                if (km < key) lo = mid + 1; else hi = mid - 1;
            }
            if (o >= 0) {
                if (DIM == 2) {
                    out[0] = w.Pk[2 * o];
                    out[1] = w.Pk[2 * o + 1];
                } else {
                    const double* q = w.Pk + 4 * o;
                    double tn = __dadd_rn(__dadd_rn(__dmul_rn(q[1], nv[0]), __dmul_rn(q[2], nv[1])),
                                          __dmul_rn(q[3], nv[2]));
                    out[0] = q[0];
                    out[1] = __dsub_rn(q[1], __dmul_rn(tn, nv[0]));
                    out[2] = __dsub_rn(q[2], __dmul_rn(tn, nv[1]));
                    out[3] = __dsub_rn(q[3], __dmul_rn(tn, nv[2]));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < pw) w.Pk_nx[pw * c + k] = out[k];   // compile-time indices keep out[] in registers
    }
}

// Geometry of a caller-supplied contact list (already in pairs_nx).
template <int DIM>
__global__ void k_geometry_given(CdGeom g, CdWork w, int nc, const double* __restrict__ pos,
                                 const double* __restrict__ radius, const double* __restrict__ inv_m,
                                 const double* __restrict__ inv_I)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int2 ab = w.pairs_nx[c];
        double nv[3], gap, mn, mt;
        contact_geometry<DIM>(g, w, ab.x, ab.y, pos, radius, inv_m, inv_I, nv, &gap, &mn, &mt);
        store_geometry<DIM>(w, c, ab.x, ab.y, nv, gap, mn, mt);
    }
}

__global__ void k_copy_pairs(int nc, const int32_t* __restrict__ src, int2* __restrict__ dst, CdCtrl* ctrl)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
        dst[c] = make_int2(src[2 * c], src[2 * c + 1]);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->nc_needed = nc;
}

// Caller-given starting impulses (or zeros) for a caller-given list.
__global__ void k_given_impulses(CdWork w, int nc, const double* __restrict__ imp, int pw)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc * pw; i += gridDim.x * blockDim.x)
        w.Pk_nx[i] = imp ? imp[i] : 0.0;
}

// The new set becomes the current one; with `n` > 0 (a detected set) the
// per-particle offsets of the detection are kept for the next warm start.
__global__ void k_commit(CdWork w, int pw, int n)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int nc = ctrl->nc_needed;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        w.pairs[c] = w.pairs_nx[c];
        for (int k = 0; k < pw; ++k) w.Pk[pw * c + k] = w.Pk_nx[pw * c + k];
    }
    if (w.poff_prev && n > 0)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + 1; i += gridDim.x * blockDim.x)
            w.poff_prev[i] = w.poff[i];
}

// by_particle: the new set's per-particle offsets are in poff_prev.
__global__ void k_set_nc(CdCtrl* ctrl, int by_particle)
{
    if (ctrl->skip) return;
    ctrl->nc = ctrl->nc_needed;
    ctrl->prev_offsets = by_particle;
}

static int grid_for(int n, int per_block = CD_BLOCK)
{
    int g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return g;
}

cudaError_t cd_launch_detect(const CdGeom& g, const CdWork& w, const double* pos, const double* radius,
                             const double* inv_m, const double* inv_I, int warm, int pw, cudaStream_t s, int* nl)
{
    int ncell = g.ncell_total;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.cell_cnt, 0, sizeof(int) * (size_t)(ncell + 1), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.cell_fill, 0, sizeof(int) * (size_t)ncell, s)) != cudaSuccess) return e;
    int gb = grid_for(g.n);
    if (g.dim == 2) k_cell_count<2><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, radius, w.cell_of, w.cell_cnt, w.ctrl);
    else k_cell_count<3><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, radius, w.cell_of, w.cell_cnt, w.ctrl);
    ++*nl;
    if ((e = cd_scan_exclusive(w.cell_cnt, w.cell_start, ncell + 1, w.scan_tmp, nullptr, s, nl)) != cudaSuccess) return e;
    k_cell_fill<<<gb, CD_BLOCK, 0, s>>>(g.n, w.cell_of, w.cell_start, w.cell_fill, w.cell_pid, w.ctrl); ++*nl;
    k_cell_sort<<<grid_for(ncell), CD_BLOCK, 0, s>>>(ncell, w.cell_start, w.cell_pid, w.ctrl); ++*nl;
    if (g.dim == 2)
        k_pair_count<2><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, radius, w.cell_of, w.cell_start, w.cell_pid, w.pcnt,
                                                w.ctrl);
    else
        k_pair_count<3><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, radius, w.cell_of, w.cell_start, w.cell_pid, w.pcnt,
                                                w.ctrl);
    ++*nl;
    if ((e = cudaMemsetAsync(w.pcnt + g.n, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cd_scan_exclusive(w.pcnt, w.poff, g.n + 1, w.scan_tmp, &w.ctrl->nc_needed, s, nl)) != cudaSuccess) return e;
    k_cap_check<<<1, 1, 0, s>>>(w.ctrl, g.cap); ++*nl;
    if (g.dim == 2) k_pair_emit<2><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, radius);
    else k_pair_emit<3><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, radius);
    ++*nl;
    int gc = grid_for(g.cap);
    if (g.dim == 2) k_geometry_warm<2><<<gc, CD_BLOCK, 0, s>>>(g, w, pos, radius, inv_m, inv_I, warm, pw);
    else k_geometry_warm<3><<<gc, CD_BLOCK, 0, s>>>(g, w, pos, radius, inv_m, inv_I, warm, pw);
    ++*nl;
    k_commit<<<gc, CD_BLOCK, 0, s>>>(w, pw, g.n); ++*nl;
    k_set_nc<<<1, 1, 0, s>>>(w.ctrl, w.poff_prev != nullptr); ++*nl;
    return cudaGetLastError();
}

cudaError_t cd_launch_set_contacts(const CdGeom& g, const CdWork& w, const double* pos, const double* radius,
                                   const double* inv_m, const double* inv_I, int nc, const int32_t* pairs,
                                   const double* impulses, int pw, cudaStream_t s, int* nl)
{
    int gc = grid_for(nc > 0 ? nc : 1);
    k_copy_pairs<<<gc, CD_BLOCK, 0, s>>>(nc, pairs, w.pairs_nx, w.ctrl); ++*nl;
    if (nc > 0) {
        if (g.dim == 2) k_geometry_given<2><<<gc, CD_BLOCK, 0, s>>>(g, w, nc, pos, radius, inv_m, inv_I);
        else k_geometry_given<3><<<gc, CD_BLOCK, 0, s>>>(g, w, nc, pos, radius, inv_m, inv_I);
        ++*nl;
    }
    k_given_impulses<<<grid_for(nc * pw > 0 ? nc * pw : 1), CD_BLOCK, 0, s>>>(w, nc, impulses, pw); ++*nl;
    k_commit<<<gc, CD_BLOCK, 0, s>>>(w, pw, 0); ++*nl;   // a caller-given list: no offsets
    k_set_nc<<<1, 1, 0, s>>>(w.ctrl, 0); ++*nl;
    return cudaGetLastError();
}
