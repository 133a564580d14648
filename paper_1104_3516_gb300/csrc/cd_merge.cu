// Merging of the last colours of a step into one sweep phase.
//
// Every colour costs a grid barrier per sweep.  Take the contacts of the M
// last colours (M = 3 or 2) and link two of them when they share a particle;
// since a particle has at most one contact of each colour, the linked groups
// ("chains": paths and cycles for M = 2, small trees and meshes for M = 3)
// are small on a dense packing, and different chains share no particle.  If
// every chain goes whole to one block of the persistent grid, the block can
// update its chains' contacts of colour K-M, synchronise its threads, update
// those of colour K-M+1, and so on: the same order as M separate phases, with
// block barriers in place of M - 1 grid barriers.
//
// Per step (after the colour order is built): label every position of the M
// colours with the smallest position of its chain (minimum propagation along
// the links, bounded rounds), count the chains, order them by label and cut
// that order into G pieces of about equal numbers of colour-(K-M) contacts
// (the largest sub-step; one piece per block), and list each block's
// positions of each colour in ascending order (one warp per list scans the
// window of positions the list spans, so the lists do not depend on timing).
// The step is merged only if the labelling converged, no chain holds more
// than 64 contacts and the last class is at most a quarter of the class
// K-M.  params.merge_last_colour 1 (or 3) tries M = 3 first and, if that is
// not taken, M = 2; 2 tries M = 2 only.  The sweep reads the decision, M or
// 0, from the control block.
#include <climits>

#include "cd_internal.cuh"

#define CD_MG_MAX_CHAIN 64
#define CD_MG_ROUNDS 80

// Colour-order positions of the M last colours: colour K-M+m at [bnd[m],
// bnd[m+1]), m = 0 .. M-1.  False when there are not at least M + 1 colours
// or one of the M classes is empty.
__device__ __forceinline__ bool mg_segment(const CdWork& w, int M, int (&bnd)[CD_MG_MAXC + 1])
{
    const int K = w.ctrl->ncolours;
    if (M < 2 || M > CD_MG_MAXC || K < M + 1 || K > CD_KMAX) return false;
    for (int m = 0; m <= M; ++m) bnd[m] = w.colour_off[K - M + m];
    for (int m = 0; m < M; ++m)
        if (bnd[m + 1] <= bnd[m]) return false;
    return true;
}

// Merged colour (0 .. M-1) of position p in [bnd[0], bnd[M]).
__device__ __forceinline__ int mg_colour(const int (&bnd)[CD_MG_MAXC + 1], int M, int p)
{
    int m = 0;
    while (m + 1 < M && p >= bnd[m + 1]) ++m;
    return m;
}

// A pass for M colours runs only if no earlier pass of this step merged
// (first: the pass that resets the decision).
__device__ __forceinline__ bool mg_pass_live(const CdCtrl* ctrl)
{
    return !ctrl->skip && ctrl->merge == 0;
}

__global__ void k_mg_init(CdGeom g, CdWork w, int M, int first)
{
    CdCtrl* ctrl = w.ctrl;
    if (!first && !mg_pass_live(ctrl)) return;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    if (first && g.merge_auto && ctrl->mg_prev > 0 && ctrl->mg_prev - 1 < CD_MG_MIN_SWEEPS) {
        // the previous solve was short: grouping the chains would cost more
        // than the barriers it saves; -1 stops this step's passes
        if (i0 == 0) ctrl->merge = -1;
        return;
    }
    for (int i = i0; i < M * g.n; i += st) w.mg_slot[i] = -1;
    const int nc = ctrl->nc;   // labels, sizes and weights are indexed by live positions only
    for (int i = i0; i <= nc; i += st) { w.mg_size[i] = 0; w.mg_w[i] = 0; }
    const int nbk = M * g.merge_blocks;
    for (int i = i0; i <= nbk; i += st) w.mg_bcnt[i] = 0;
    for (int i = i0; i < nbk; i += st) { w.mg_bmin[i] = INT_MAX; w.mg_bmax[i] = -1; }
    if (i0 == 0) {
        if (first) ctrl->merge = 0;
        ctrl->mg_changed = 1;
        ctrl->mg_maxsize = 0;
    }
}

__global__ void k_mg_mark(CdGeom g, CdWork w, int M)
{
    if (!mg_pass_live(w.ctrl)) return;
    int bnd[CD_MG_MAXC + 1];
    if (!mg_segment(w, M, bnd)) return;
    for (int p = bnd[0] + blockIdx.x * blockDim.x + threadIdx.x; p < bnd[M]; p += gridDim.x * blockDim.x) {
        const int2 ab = w.c_ab[p];
        int* slot = w.mg_slot + mg_colour(bnd, M, p) * g.n;
        slot[ab.x] = p;
        if (ab.y < g.n) slot[ab.y] = p;
        w.mg_label[p] = p;
    }
}

// Minimum propagation along the links, one round per grid barrier, until no
// label moves (labels only decrease, so reading a neighbour's label while it
// changes is harmless).  round_cnt (free after the colouring) holds three
// rotating "moved" flags.
__global__ void k_mg_label(CdGeom g, CdWork w, int* flag, int M)
{
    CdCtrl* ctrl = w.ctrl;
    if (!mg_pass_live(ctrl)) return;
    int bnd[CD_MG_MAXC + 1];
    if (!mg_segment(w, M, bnd)) return;
    const unsigned long long nb = gridDim.x;
    unsigned long long epoch = 0;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    if (tid == 0) { flag[0] = 0; flag[1] = 0; flag[2] = 0; }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    for (int round = 0; round < CD_MG_ROUNDS; ++round) {
        // round r writes flag r % 3 before its barrier and everyone reads it after;
        // flag (r + 1) % 3 was last read before the previous barrier
        if (tid == 0) flag[(round + 1) % 3] = 0;
        int moved = 0;
        for (int p = bnd[0] + tid; p < bnd[M]; p += st) {
            const int2 ab = w.c_ab[p];
            const int mp = mg_colour(bnd, M, p);
            int m = cd_ld_volatile_int(&w.mg_label[p]);
            const int own = m;
            for (int q = 0; q < M; ++q) {
                if (q == mp) continue;
                const int* other = w.mg_slot + q * g.n;
                const int d0 = other[ab.x];
                if (d0 >= 0) m = min(m, cd_ld_volatile_int(&w.mg_label[d0]));
                if (ab.y < g.n) {
                    const int d1 = other[ab.y];
                    if (d1 >= 0) m = min(m, cd_ld_volatile_int(&w.mg_label[d1]));
                }
            }
            if (m < own) {
                *(volatile int*)&w.mg_label[p] = m;
                moved = 1;
            }
        }
        if (__syncthreads_or(moved) && threadIdx.x == 0) atomicExch(&flag[round % 3], 1);
        if (!cd_grid_sync(ctrl, nb, epoch)) return;
        if (cd_ld_volatile_int(&flag[round % 3]) == 0) {
            if (tid == 0) ctrl->mg_changed = 0;   // converged
            return;
        }
    }
}

// Chain sizes (all contacts, for the size limit) and weights (contacts of
// colour K-M, which the pieces balance).
__global__ void k_mg_size(CdGeom g, CdWork w, int M)
{
    if (!mg_pass_live(w.ctrl)) return;
    int bnd[CD_MG_MAXC + 1];
    if (!mg_segment(w, M, bnd)) return;
    for (int p = bnd[0] + blockIdx.x * blockDim.x + threadIdx.x; p < bnd[M]; p += gridDim.x * blockDim.x) {
        const int lab = w.mg_label[p];
        const int s = atomicAdd(&w.mg_size[lab], 1) + 1;
        atomicMax(&w.ctrl->mg_maxsize, s);
        if (p < bnd[1]) atomicAdd(&w.mg_w[lab], 1);
    }
}

// The decision, then each position's bucket m G + block: chains in label
// order cut into G pieces of about equal colour-(K-M) counts.
__global__ void k_mg_bucket(CdGeom g, CdWork w, int M)
{
    CdCtrl* ctrl = w.ctrl;
    if (!mg_pass_live(ctrl)) return;
    int bnd[CD_MG_MAXC + 1];
    if (!mg_segment(w, M, bnd)) return;
    const bool ok = ctrl->mg_changed == 0 && ctrl->mg_maxsize <= CD_MG_MAX_CHAIN &&
                    4 * (bnd[M] - bnd[M - 1]) <= (bnd[1] - bnd[0]);
    if (!ok) return;
    const int G = g.merge_blocks;
    const long long total = bnd[1] - bnd[0];
    for (int p = bnd[0] + blockIdx.x * blockDim.x + threadIdx.x; p < bnd[M]; p += gridDim.x * blockDim.x) {
        const long long off = w.mg_start[w.mg_label[p]];   // colour-(K-M) contacts of the chains before
        int blk = (int)((off * G) / total);
        if (blk > G - 1) blk = G - 1;
        const int k = mg_colour(bnd, M, p) * G + blk;
        w.mg_bucket[p] = k;
        atomicAdd(&w.mg_bcnt[k], 1);
        atomicMin(&w.mg_bmin[k], p);
        atomicMax(&w.mg_bmax[k], p);
    }
}

// Publishes the decision after every block of k_mg_bucket has run (a kernel
// of its own: the bucket kernel's blocks read ctrl->merge through
// mg_pass_live while they work).
__global__ void k_mg_decide(CdWork w, int M)
{
    CdCtrl* ctrl = w.ctrl;
    if (!mg_pass_live(ctrl)) return;
    int bnd[CD_MG_MAXC + 1];
    if (!mg_segment(w, M, bnd)) return;
    const bool ok = ctrl->mg_changed == 0 && ctrl->mg_maxsize <= CD_MG_MAX_CHAIN &&
                    4 * (bnd[M] - bnd[M - 1]) <= (bnd[1] - bnd[0]);
    if (ok) ctrl->merge = M;
}

// One warp per bucket lists its positions in ascending order.
__global__ void k_mg_fill(CdGeom g, CdWork w, int M)
{
    if (w.ctrl->skip || w.ctrl->merge != M) return;
    const int lane = threadIdx.x & 31;
    const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= M * g.merge_blocks) return;
    const int lo = w.mg_bmin[k], hi = w.mg_bmax[k];
    int base = w.mg_boff[k];
    for (int p0 = lo; p0 <= hi; p0 += 32) {
        const int p = p0 + lane;
        const bool mem = p <= hi && w.mg_bucket[p] == k;
        const unsigned m = __ballot_sync(0xffffffffu, mem);
        if (mem) w.mg_list[base + __popc(m & ((1u << lane) - 1u))] = p;
        base += __popc(m);
    }
}

// One pass of the pipeline for M colours.
static cudaError_t merge_pass(const CdGeom& g, const CdWork& w, int coop_blocks, int M, int first, cudaStream_t s,
                              int* nl)
{
    cudaError_t e;
    const int nbk = M * g.merge_blocks;
    int m = g.cap + 1;
    if (M * g.n > m) m = M * g.n;
    if (nbk + 1 > m) m = nbk + 1;
    int gm = (m + CD_BLOCK - 1) / CD_BLOCK;
    if (gm > 4096) gm = 4096;
    int gc = (g.cap + CD_BLOCK - 1) / CD_BLOCK;
    if (gc < 1) gc = 1;
    if (gc > 4096) gc = 4096;
    k_mg_init<<<gm, CD_BLOCK, 0, s>>>(g, w, M, first);
    k_mg_mark<<<gc, CD_BLOCK, 0, s>>>(g, w, M);
    *nl += 2;
    {
        CdGeom ga = g;
        CdWork wa = w;
        int* flag = w.round_cnt;
        int mm = M;
        void* args[] = {&ga, &wa, &flag, &mm};
        if ((e = cudaMemsetAsync(w.ctrl, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
        if ((e = cudaLaunchCooperativeKernel((const void*)k_mg_label, dim3(coop_blocks), dim3(CD_SWEEP_THREADS), args, 0,
                                             s)) != cudaSuccess)
            return e;
        ++*nl;
    }
    k_mg_size<<<gc, CD_BLOCK, 0, s>>>(g, w, M);
    ++*nl;
    // the live contacts only (their count read on the device)
    if ((e = cd_scan_exclusive(w.mg_w, w.mg_start, g.cap + 1, w.scan_tmp, nullptr, s, nl, &w.ctrl->nc)) != cudaSuccess)
        return e;
    k_mg_bucket<<<gc, CD_BLOCK, 0, s>>>(g, w, M);
    k_mg_decide<<<1, 1, 0, s>>>(w, M);
    *nl += 2;
    if ((e = cd_scan_exclusive(w.mg_bcnt, w.mg_boff, nbk + 1, w.scan_tmp, nullptr, s, nl)) != cudaSuccess) return e;
    k_mg_fill<<<(nbk * 32 + 255) / 256, 256, 0, s>>>(g, w, M);
    ++*nl;
    return cudaGetLastError();
}

// The passes run in turn on the stream; a pass after one that merged does
// nothing but its two scans, which recompute the same offsets from the
// unchanged counts (the first M G + 1 bucket counts and the chain weights).
cudaError_t cd_launch_merge(const CdGeom& g, const CdWork& w, int coop_blocks, cudaStream_t s, int* nl)
{
    cudaError_t e;
    const int mmax = (g.merge_last == 2) ? 2 : CD_MG_MAXC;
    for (int M = mmax; M >= 2; --M)
        if ((e = merge_pass(g, w, coop_blocks, M, M == mmax, s, nl)) != cudaSuccess) return e;
    return cudaSuccess;
}

int cd_merge_label_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mg_label, CD_SWEEP_THREADS, 0) != cudaSuccess) return 0;
    return b;
}
