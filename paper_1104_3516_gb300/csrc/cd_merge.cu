// Merging of the two last colours of a step into one sweep phase.
//
// Every colour costs a grid barrier per sweep; after the colour repair the
// last class of a dense packing is small (2,293 of 223,196 contacts on the
// 1e5-disc pile) but still a whole phase.  The contacts of the second-last
// colour (A) and of the last colour (B) form chains: an A contact and a B
// contact are linked when they share a particle, and since a particle has at
// most one contact of each colour, a chain is a path or a cycle alternating
// A and B.  Different chains share no particle.  If every chain goes whole
// to one block of the persistent grid, the block can update its chains' A
// contacts, synchronise its threads and then update their B contacts: the
// same order as the two phases, with a block barrier in place of a grid
// barrier.
//
// Per step (after the colour order is built): label every position of the
// two colours with the smallest position of its chain (minimum propagation
// along the links, bounded rounds), count the chains, order them by label
// and cut that order into G pieces of about equal contact counts (one per
// block), and list each block's A positions and B positions in ascending
// order (one warp per list scans the window of positions the list spans, so
// the lists do not depend on timing).  The step is merged only if the
// labelling converged, no chain holds more than 64 contacts and the B class
// is at most a quarter of the A class; the sweep reads the decision from the
// control block.
#include <climits>

#include "cd_internal.cuh"

#define CD_MG_MAX_CHAIN 64
#define CD_MG_ROUNDS 80

// Positions [a0, b0) hold the second-last colour, [b0, e) the last one.
__device__ __forceinline__ bool mg_segment(const CdWork& w, int& a0, int& b0, int& e)
{
    const int K = w.ctrl->ncolours;
    if (K < 3 || K > CD_KMAX) return false;
    a0 = w.colour_off[K - 2];
    b0 = w.colour_off[K - 1];
    e = w.colour_off[K];
    return b0 > a0 && e > b0;
}

__global__ void k_mg_init(CdGeom g, CdWork w)
{
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    for (int i = i0; i < g.n; i += st) { w.mg_pa[i] = -1; w.mg_pb[i] = -1; }
    for (int i = i0; i <= g.cap; i += st) w.mg_size[i] = 0;
    const int nbk = 2 * g.merge_blocks;
    for (int i = i0; i <= nbk; i += st) w.mg_bcnt[i] = 0;
    for (int i = i0; i < nbk; i += st) { w.mg_bmin[i] = INT_MAX; w.mg_bmax[i] = -1; }
    if (i0 == 0) {
        w.ctrl->merge = 0;
        w.ctrl->mg_changed = 1;
        w.ctrl->mg_maxsize = 0;
    }
}

__global__ void k_mg_mark(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    int a0, b0, e;
    if (!mg_segment(w, a0, b0, e)) return;
    for (int p = a0 + blockIdx.x * blockDim.x + threadIdx.x; p < e; p += gridDim.x * blockDim.x) {
        const int2 ab = w.c_ab[p];
        int* slot = (p < b0) ? w.mg_pa : w.mg_pb;
        slot[ab.x] = p;
        if (ab.y < g.n) slot[ab.y] = p;
        w.mg_label[p] = p;
    }
}

// Minimum propagation along the links, one round per grid barrier, until no
// label moves (labels only decrease, so reading a neighbour's label while it
// changes is harmless).  round_cnt (free after the colouring) holds three
// rotating "moved" flags.
__global__ void k_mg_label(CdGeom g, CdWork w, int* flag)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int a0, b0, e;
    if (!mg_segment(w, a0, b0, e)) return;
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
        for (int p = a0 + tid; p < e; p += st) {
            const int2 ab = w.c_ab[p];
            const int* other = (p < b0) ? w.mg_pb : w.mg_pa;
            int m = cd_ld_volatile_int(&w.mg_label[p]);
            const int own = m;
            const int d0 = other[ab.x];
            if (d0 >= 0) m = min(m, cd_ld_volatile_int(&w.mg_label[d0]));
            if (ab.y < g.n) {
                const int d1 = other[ab.y];
                if (d1 >= 0) m = min(m, cd_ld_volatile_int(&w.mg_label[d1]));
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

__global__ void k_mg_size(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    int a0, b0, e;
    if (!mg_segment(w, a0, b0, e)) return;
    for (int p = a0 + blockIdx.x * blockDim.x + threadIdx.x; p < e; p += gridDim.x * blockDim.x) {
        const int s = atomicAdd(&w.mg_size[w.mg_label[p]], 1) + 1;
        atomicMax(&w.ctrl->mg_maxsize, s);
    }
}

// The decision, then each position's bucket: chains in label order cut into
// G pieces of about equal size.
__global__ void k_mg_bucket(CdGeom g, CdWork w)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int a0, b0, e;
    if (!mg_segment(w, a0, b0, e)) return;
    const bool ok = ctrl->mg_changed == 0 && ctrl->mg_maxsize <= CD_MG_MAX_CHAIN && 4 * (e - b0) <= (b0 - a0);
    if (!ok) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->merge = 1;
    const int G = g.merge_blocks;
    const long long total = e - a0;
    for (int p = a0 + blockIdx.x * blockDim.x + threadIdx.x; p < e; p += gridDim.x * blockDim.x) {
        const long long off = w.mg_start[w.mg_label[p]];   // chains before this one, in label order
        int blk = (int)((off * G) / total);
        if (blk > G - 1) blk = G - 1;
        const int k = (p < b0) ? blk : G + blk;
        w.mg_bucket[p] = k;
        atomicAdd(&w.mg_bcnt[k], 1);
        atomicMin(&w.mg_bmin[k], p);
        atomicMax(&w.mg_bmax[k], p);
    }
}

// One warp per bucket lists its positions in ascending order.
__global__ void k_mg_fill(CdGeom g, CdWork w)
{
    if (w.ctrl->skip || !w.ctrl->merge) return;
    const int lane = threadIdx.x & 31;
    const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= 2 * g.merge_blocks) return;
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

cudaError_t cd_launch_merge(const CdGeom& g, const CdWork& w, int coop_blocks, cudaStream_t s, int* nl)
{
    cudaError_t e;
    const int nbk = 2 * g.merge_blocks;
    int m = g.cap + 1;
    if (g.n > m) m = g.n;
    if (nbk + 1 > m) m = nbk + 1;
    int gm = (m + CD_BLOCK - 1) / CD_BLOCK;
    if (gm > 4096) gm = 4096;
    int gc = (g.cap + CD_BLOCK - 1) / CD_BLOCK;
    if (gc < 1) gc = 1;
    if (gc > 4096) gc = 4096;
    k_mg_init<<<gm, CD_BLOCK, 0, s>>>(g, w);
    k_mg_mark<<<gc, CD_BLOCK, 0, s>>>(g, w);
    *nl += 2;
    {
        CdGeom ga = g;
        CdWork wa = w;
        int* flag = w.round_cnt;
        void* args[] = {&ga, &wa, &flag};
        if ((e = cudaMemsetAsync(w.ctrl, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
        if ((e = cudaLaunchCooperativeKernel((const void*)k_mg_label, dim3(coop_blocks), dim3(CD_SWEEP_THREADS), args, 0,
                                             s)) != cudaSuccess)
            return e;
        ++*nl;
    }
    k_mg_size<<<gc, CD_BLOCK, 0, s>>>(g, w);
    ++*nl;
    if ((e = cd_scan_exclusive(w.mg_size, w.mg_start, g.cap + 1, w.scan_tmp, nullptr, s, nl)) != cudaSuccess) return e;
    k_mg_bucket<<<gc, CD_BLOCK, 0, s>>>(g, w);
    ++*nl;
    if ((e = cd_scan_exclusive(w.mg_bcnt, w.mg_boff, nbk + 1, w.scan_tmp, nullptr, s, nl)) != cudaSuccess) return e;
    k_mg_fill<<<(nbk * 32 + 255) / 256, 256, 0, s>>>(g, w);
    ++*nl;
    return cudaGetLastError();
}

int cd_merge_label_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mg_label, CD_SWEEP_THREADS, 0) != cudaSuccess) return 0;
    return b;
}
