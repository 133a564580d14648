// cd_colour.cu -- colouring of the contact graph and the colour ordering.
//
// The paper updates contacts one by one in random order (Sec. 2.1).  On the
// GPU the same nonlinear Gauss-Seidel runs in a colour order: contacts that
// share no particle are independent, so one colour class is updated in
// parallel and every freshly computed impulse is seen by the later colours.
//
// Colouring: Jones-Plassmann with priority (d_a + d_b) * 2^56 +
// (splitmix64(seed ^ key) >> 8), d the contacts of a particle (largest degree
// first, which needs one colour fewer than a random order on dense piles),
// ties by ascending key.  A contact takes the smallest colour not used by any
// higher-priority neighbour once all of those are coloured; the fixed point
// equals the greedy colouring in descending priority, so the result does not
// depend on scheduling.  Walls never conflict.
//
// Ordering: stable partition of the key-ordered contacts by colour (chunk
// histograms, one exclusive scan, a rank within the chunk from warp match
// masks), then the contact data is gathered into colour order in the sweep's
// real type.
#include <type_traits>

#include "cd_internal.cuh"

__global__ void k_p2c_count(CdGeom g, CdWork w)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int nc = ctrl->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int2 ab = w.pairs[c];
        atomicAdd(&w.p2c_cnt[ab.x], 1);
        if (cd_is_body(g, ab.y)) atomicAdd(&w.p2c_cnt[ab.y], 1);
    }
}

__global__ void k_p2c_fill(CdGeom g, CdWork w)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int nc = ctrl->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int2 ab = w.pairs[c];
        int s = atomicAdd(&w.p2c_fill[ab.x], 1);
        w.p2c[w.p2c_off[ab.x] + s] = c;
        if (cd_is_body(g, ab.y)) {
            s = atomicAdd(&w.p2c_fill[ab.y], 1);
            w.p2c[w.p2c_off[ab.y] + s] = c;
        }
    }
}

// Each particle's contact list in ascending key order (the atomic fill leaves
// it in arrival order); makes every later per-particle accumulation
// deterministic.
__global__ void k_p2c_sort(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    const int nbody = g.n + (g.dyn_walls ? 6 : 0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbody; i += gridDim.x * blockDim.x) {
        int b = w.p2c_off[i], e = w.p2c_off[i + 1];
        for (int k = b + 1; k < e; ++k) {
            int v = w.p2c[k];
            int j = k - 1;
            while (j >= b && w.p2c[j] > v) { w.p2c[j + 1] = w.p2c[j]; --j; }
            w.p2c[j + 1] = v;
        }
    }
}

// Persistent cooperative kernel: Jones-Plassmann rounds separated by the
// bounded grid barrier.  `prio` scratch lives in the chunk buffer (8 bytes per
// contact is reserved there by the workspace layout).
//
// Worklist form: every contact first counts its neighbours of higher
// priority (contacts sharing a body); those with
// none start the first list.  A round colours the contacts of its list (the
// smallest colour no higher-priority neighbour has; all of those are
// coloured by then) and decrements the counts of their lower-priority
// neighbours; a contact whose count reaches zero joins the next list.  Each
// contact is coloured exactly once, from the same neighbours as in the
// round-by-round scan, so the colouring is the same greedy fixed point, at a
// cost proportional to the contacts and their neighbours instead of to
// rounds x contacts.  Scratch: the colour repair's arrays (used only after
// the colouring): rep_flag holds the counts, rep_list and rep_path the lists
// of even and odd rounds; round_cnt[r % 3] is the length of round r's list
// (three counters, so that one grid barrier per round suffices: round r
// clears the counter of round r + 2, last read in round r - 1).
__device__ __forceinline__ bool jp_higher(const CdWork& w, const unsigned long long* prio, int d, int c,
                                          unsigned long long pc, unsigned long long kc)
{
    const unsigned long long pd = prio[d];
    if (pd != pc) return pd > pc;
    const int2 dd = w.pairs[d];
    return cd_key(dd.x, dd.y) < kc;
}

// Appends c to list (length at *len) with one atomic per warp.
__device__ __forceinline__ void jp_append(int* list, int* len, int c, bool take)
{
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(len, __popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (take) list[base + __popc(m & ((1u << lane) - 1u))] = c;
}

// Appends each lane's up to four entries c[u] (take[u]) with one atomic per
// warp: the lane's offset is the exclusive prefix sum of the lanes' counts.
__device__ __forceinline__ void jp_append4(int* list, int* len, const int (&c)[4], const bool (&take)[4])
{
    const int lane = threadIdx.x & 31;
    int k = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) k += take[u] ? 1 : 0;
    int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    int base = 0;
    if (lane == 31) base = atomicAdd(len, total);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - k;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (take[u]) list[base++] = c[u];
}

__global__ void __launch_bounds__(CD_SWEEP_THREADS) k_jp(CdGeom g, CdWork w, unsigned long long* prio,
                                                          int* round_cnt)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    const int nc = ctrl->nc;
    const unsigned long long nb = gridDim.x;
    unsigned long long epoch = 0;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    int* cnt = w.rep_flag;
    for (int c = tid; c < nc; c += stride) {
        int2 ab = w.pairs[c];
        unsigned long long h;
        if (g.npk > 1) {
            // a packing of a batch is coloured with its own seed and local
            // ids (walls n_b + k), exactly as if it were a system alone
            const CdPack& P = w.pk[w.pack_of[ab.x]];
            const int al = ab.x - P.first;
            const int bl = (ab.y < g.n) ? ab.y - P.first : P.count + (ab.y - g.n) % 6;
            h = cd_splitmix64(P.seed ^ cd_key(al, bl));
        } else {
            h = cd_splitmix64(g.seed ^ cd_key(ab.x, ab.y));
        }
        // largest degree first (contacts of both ends, capped at 255), then the hash
        unsigned long long ds = (unsigned long long)(w.p2c_off[ab.x + 1] - w.p2c_off[ab.x]);
        if (cd_is_body(g, ab.y)) ds += (unsigned long long)(w.p2c_off[ab.y + 1] - w.p2c_off[ab.y]);
        if (ds > 255ULL) ds = 255ULL;
        prio[c] = (ds << 56) | (h >> 8);
        w.colour[c] = -1;
    }
    if (tid == 0) { round_cnt[0] = 0; round_cnt[1] = 0; round_cnt[2] = 0; ctrl->ncolours = 0; }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    // higher-priority neighbours of every contact; the free ones start the first list
    for (int c0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < nc; c0 += stride) {
        const int c = c0 + (threadIdx.x & 31);
        int k = 0;
        if (c < nc) {
            const unsigned long long pc = prio[c];
            const int2 ab = w.pairs[c];
            const unsigned long long kc = cd_key(ab.x, ab.y);
            for (int side = 0; side < 2; ++side) {
                const int q = side ? ab.y : ab.x;
                if (!cd_is_body(g, q)) continue;
                const int f0 = w.p2c_off[q], f1 = w.p2c_off[q + 1];
                for (int t = f0; t < f1; t += 4) {
                    int d[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) d[u] = (t + u < f1) ? w.p2c[t + u] : -1;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (d[u] >= 0 && d[u] != c &&
                            jp_higher(w, prio, d[u], c, pc, kc))
                            ++k;
                }
            }
            cnt[c] = k;
        }
        jp_append(w.rep_list, &round_cnt[0], c, c < nc && k == 0);   // round 0's list
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    for (int round = 0; round < (1 << 20); ++round) {
        // even rounds read rep_list and fill rep_path, odd rounds the reverse
        // (selected, not indexed: an indexed pair of pointers lives in local memory)
        int* const list_cur = (round & 1) ? w.rep_path : w.rep_list;
        int* const list_nxt = (round & 1) ? w.rep_list : w.rep_path;
        const int len = cd_ld_volatile_int(&round_cnt[round % 3]);
        if (len == 0) break;
        if (tid == 0) round_cnt[(round + 2) % 3] = 0;
        for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < len; i0 += stride) {
            const int i = i0 + (threadIdx.x & 31);
            const int c = (i < len) ? list_cur[i] : -1;
            int2 ab = make_int2(0, 0);
            unsigned long long pc = 0ULL, kc = 0ULL;
            if (c >= 0) {
                pc = prio[c];
                ab = w.pairs[c];
                kc = cd_key(ab.x, ab.y);
            }
            // one pass over both bodies' contacts: the colours of the higher-priority
            // neighbours (all final), and the release of the lower-priority ones (they
            // read c's colour only in a later round, after the grid barrier)
            unsigned long long used = 0ULL;
            for (int side = 0; side < 2; ++side) {
                const int q = side ? ab.y : ab.x;
                const bool on = c >= 0 && cd_is_body(g, q);
                const int f0 = on ? w.p2c_off[q] : 0, f1 = on ? w.p2c_off[q + 1] : 0;
                int most = f1 - f0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) most = max(most, __shfl_xor_sync(0xffffffffu, most, o));
                // four neighbours at a time: their loads and atomics are in flight together
                for (int t = 0; t < most; t += 4) {
                    int d[4], v[4];
                    bool hi[4], lo[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) d[u] = (f0 + t + u < f1) ? w.p2c[f0 + t + u] : -1;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool nb_ok = d[u] >= 0 && d[u] != c;
                        const bool h = nb_ok && jp_higher(w, prio, d[u], c, pc, kc);
                        hi[u] = h;
                        lo[u] = nb_ok && !h;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = hi[u] ? cd_ld_volatile_int(&w.colour[d[u]]) : (lo[u] ? atomicSub(&cnt[d[u]], 1) : 0);
                    bool rel[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (hi[u] && v[u] >= 0) used |= 1ULL << v[u];
                        rel[u] = lo[u] && v[u] == 1;   // its last higher-priority neighbour: next round
                    }
                    jp_append4(list_nxt, &round_cnt[(round + 1) % 3], d, rel);
                }
            }
            int top = 0;
            if (c >= 0) {
                const int col = (used == ~0ULL) ? 64 : __ffsll((long long)~used) - 1;
                if (col >= CD_KMAX) {
                    atomicCAS(&ctrl->error, CDE_NONE, CDE_COLOURS);
                } else {
                    *(volatile int*)&w.colour[c] = col;
                    top = col + 1;
                }
            }
            top = __reduce_max_sync(0xffffffffu, top);   // one atomic per warp
            if ((threadIdx.x & 31) == 0 && top > 0) atomicMax(&ctrl->ncolours, top);
        }
        if (!cd_grid_sync(ctrl, nb, epoch)) return;
        if (cd_ld_volatile_int(&ctrl->error) != CDE_NONE) break;
    }
}

// ---------------------------------------------------------------------------
// Repair of the highest colour (Kempe chains; the recolouring step of the
// classical proof of Vizing's theorem, used as a heuristic).  For each
// packing (a plain system is one): if its greedy colouring has a colour more
// than its busiest body has contacts, and that top colour T holds at most
// max(1, min(1024, nc_b / 256)) contacts, one warp visits them in key
// order.  Contact c = (u, v) takes the smallest colour below T that neither
// u nor v has; failing that, for a free at u and b free at v (ascending),
// the path leaving v on its colour-a contact and alternating a, b is
// followed to its end (a body without the next colour, or a wall); unless it
// reaches u, a and b are swapped along it and c takes a.  Fewer colours mean
// fewer grid barriers per sweep.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rep_pack_of(const CdGeom& g, const CdWork& w, int body)
{
    return (g.npk > 1) ? w.pack_of[body] : 0;
}

__global__ void k_rep_init(CdGeom g, CdWork w)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < g.npk; b += gridDim.x * blockDim.x) {
        w.rep_top[b] = -1;
        w.rep_dmax[b] = 0;
    }
}

// atomicMax of v into dst[key], one atomic per run of lanes with the same key
// (the plain system's single packing would otherwise serialise every
// contact on one address).
__device__ __forceinline__ void warp_atomic_max(int* dst, int key, int v, bool active)
{
    const unsigned grp = __match_any_sync(0xffffffffu, active ? key : -1);
    const int m = __reduce_max_sync(grp, active ? v : -1);
    if (active && (threadIdx.x & 31) == __ffs(grp) - 1) atomicMax(&dst[key], m);
}

__global__ void k_rep_scan_colours(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    const int nc = w.ctrl->nc;
    const int nbody = g.n + (g.dyn_walls ? 6 : 0);
    const int st = gridDim.x * blockDim.x;
    // whole warps iterate together (the warp collectives need every lane)
    for (int c0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < nc; c0 += st) {
        const int c = c0 + (threadIdx.x & 31);
        const bool on = c < nc;
        warp_atomic_max(w.rep_top, on ? rep_pack_of(g, w, w.pairs[c].x) : 0, on ? w.colour[c] : -1, on);
    }
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < nbody; i0 += st) {
        const int i = i0 + (threadIdx.x & 31);
        const bool on = i < nbody;
        const int pk = (on && i < g.n) ? rep_pack_of(g, w, i) : 0;
        warp_atomic_max(w.rep_dmax, pk, on ? w.p2c_off[i + 1] - w.p2c_off[i] : 0, on);
    }
}

// Flags over the whole capacity (the scan runs over cap + 1 entries).
__global__ void k_rep_flag(CdGeom g, CdWork w)
{
    if (w.ctrl->skip) return;
    const int nc = w.ctrl->nc;
    // up to nc: the scan of the flags reads the live contacts only
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= nc; c += gridDim.x * blockDim.x) {
        int f = 0;
        if (c < nc) {
            const int t = w.rep_top[rep_pack_of(g, w, w.pairs[c].x)];
            f = (t > 0 && w.colour[c] == t) ? 1 : 0;
        }
        w.rep_flag[c] = f;
    }
}

__global__ void k_rep_fill(CdWork w)
{
    if (w.ctrl->skip) return;
    const int nc = w.ctrl->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
        if (w.rep_flag[c]) w.rep_list[w.rep_pos[c]] = c;
}

// The repair runs one warp per packing: every step is sequential, but the
// lanes read a body's contact list together, so a step costs a few L2 round
// trips instead of one per contact of the body.  All lanes follow the same
// control flow; lane 0 writes.

// Colours below t that body x has on no contact other than c (all of them
// for a wall that is not a body).
__device__ __forceinline__ unsigned long long rep_free(const CdGeom& g, const CdWork& w, int x, int c, int t)
{
    const unsigned long long all = (1ULL << t) - 1ULL;
    if (!cd_is_body(g, x)) return all;
    const int lane = threadIdx.x & 31;
    const int f0 = w.p2c_off[x], f1 = w.p2c_off[x + 1];
    unsigned long long used = 0ULL;
    for (int f = f0; f < f1; f += 32) {
        unsigned long long bit = 0ULL;
        if (f + lane < f1) {
            const int d = w.p2c[f + lane];
            const int k = w.colour[d];
            if (d != c && k >= 0 && k < t) bit = 1ULL << k;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bit |= __shfl_xor_sync(0xffffffffu, bit, o);
        used |= bit;
    }
    return all & ~used;
}

// Body x's contact of colour cur (at most one in a proper colouring), or -1.
__device__ __forceinline__ int rep_find(const CdWork& w, int x, int cur)
{
    const int lane = threadIdx.x & 31;
    const int f0 = w.p2c_off[x], f1 = w.p2c_off[x + 1];
    for (int f = f0; f < f1; f += 32) {
        int d = -1;
        if (f + lane < f1) {
            const int dd = w.p2c[f + lane];
            if (w.colour[dd] == cur) d = dd;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, d >= 0);
        if (hit) return __shfl_sync(0xffffffffu, d, __ffs(hit) - 1);
    }
    return -1;
}

__global__ void k_rep_run(CdGeom g, CdWork w)
{
    if (w.ctrl->skip || w.ctrl->error != CDE_NONE) return;   // e.g. an uncoloured contact
    const int nc = w.ctrl->nc;
    const int lane = threadIdx.x & 31;
    const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);   // one warp per packing
    if (b >= g.npk) return;
    const int c0 = (g.npk > 1) ? w.pk_coff[b] : 0, c1 = (g.npk > 1) ? w.pk_coff[b + 1] : nc;
    const int ncb = c1 - c0, t = w.rep_top[b];
    if (ncb <= 0 || t <= 0 || t > 63 || t + 1 <= w.rep_dmax[b]) return;
    const int l0 = w.rep_pos[c0], l1 = w.rep_pos[c1];
    int limit = ncb / 256;
    if (limit > 1024) limit = 1024;
    if (limit < 1) limit = 1;
    if (l1 - l0 > limit) return;
    int* path = w.rep_path + c0;
    for (int l = l0; l < l1; ++l) {
        const int c = w.rep_list[l];
        const int2 uv = w.pairs[c];
        const int u = uv.x, v = uv.y;
        const unsigned long long mu = rep_free(g, w, u, c, t), mv = rep_free(g, w, v, c, t);
        if (mu & mv) {
            if (lane == 0) w.colour[c] = __ffsll((long long)(mu & mv)) - 1;
            __syncwarp();
            continue;
        }
        if (!cd_is_body(g, v)) continue;
        bool done = false;
        for (int a = 0; a < t && !done; ++a) {
            if (!((mu >> a) & 1ULL)) continue;
            for (int bb = 0; bb < t && !done; ++bb) {
                if (!((mv >> bb) & 1ULL)) continue;
                int len = 0, x = v, cur = a;
                bool fail = false;
                for (;;) {
                    const int e = rep_find(w, x, cur);
                    if (e < 0) break;
                    const int2 pe = w.pairs[e];
                    const int y = (pe.x == x) ? pe.y : pe.x;
                    if (lane == 0) path[len] = e;
                    ++len;
                    if (y == u) { fail = true; break; }
                    if (!cd_is_body(g, y)) break;
                    x = y;
                    cur = (cur == a) ? bb : a;
                    if (len >= ncb) { fail = true; break; }
                }
                __syncwarp();
                if (fail) continue;
                for (int i = lane; i < len; i += 32) {
                    const int e = path[i];
                    w.colour[e] = (w.colour[e] == a) ? bb : a;
                }
                if (lane == 0) w.colour[c] = a;
                __syncwarp();
                done = true;
            }
        }
    }
}

__global__ void k_rep_ncolours_reset(CdCtrl* ctrl)
{
    if (!ctrl->skip) ctrl->ncolours = 0;
}

__global__ void k_rep_ncolours(CdWork w)
{
    if (w.ctrl->skip) return;
    const int nc = w.ctrl->nc;
    // warps step together (uniform bound); one atomic per warp
    for (int c0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < nc; c0 += gridDim.x * blockDim.x) {
        const int c = c0 + (threadIdx.x & 31);
        const int top = __reduce_max_sync(0xffffffffu, c < nc ? w.colour[c] + 1 : 0);
        if ((threadIdx.x & 31) == 0) atomicMax(&w.ctrl->ncolours, top);
    }
}

static cudaError_t launch_repair(const CdGeom& g, const CdWork& w, int gc, cudaStream_t s, int* nl)
{
    cudaError_t e;
    const int gp = (g.npk + CD_BLOCK - 1) / CD_BLOCK;
    int m = (g.cap > g.n + 6) ? g.cap : g.n + 6;
    int gm = (m + CD_BLOCK - 1) / CD_BLOCK;
    if (gm > 4096) gm = 4096;
    k_rep_init<<<gp, CD_BLOCK, 0, s>>>(g, w);
    k_rep_scan_colours<<<gm, CD_BLOCK, 0, s>>>(g, w);
    k_rep_flag<<<gc, CD_BLOCK, 0, s>>>(g, w);
    *nl += 3;
    // the live contacts only (their count read on the device)
    if ((e = cd_scan_exclusive(w.rep_flag, w.rep_pos, g.cap + 1, w.scan_tmp, nullptr, s, nl, &w.ctrl->nc)) !=
        cudaSuccess)
        return e;
    k_rep_fill<<<gc, CD_BLOCK, 0, s>>>(w);
    // one warp per packing: a plain system's repair is one sequential walk
    k_rep_run<<<(g.npk + 1) / 2, 64, 0, s>>>(g, w);
    k_rep_ncolours_reset<<<1, 1, 0, s>>>(w.ctrl);
    k_rep_ncolours<<<gc, CD_BLOCK, 0, s>>>(w);
    *nl += 4;
    return cudaGetLastError();
}

// Per-chunk colour histogram, layout [colour][chunk].
// Chunks of CD_CHUNK colour-order positions: only the live ones (those
// holding contacts) are counted, laid out [colour][live chunk], and scanned.
__device__ __forceinline__ int live_chunks(int nc) { return (nc + CD_CHUNK - 1) / CD_CHUNK; }

__global__ void k_chunk_hist(CdWork w)
{
    __shared__ int s_cnt[CD_KMAX];
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int nc = ctrl->nc;
    const int ncl = live_chunks(nc);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->chunk_last = CD_KMAX * ncl - 1;
    if ((int)blockIdx.x >= ncl) return;
    for (int k = threadIdx.x; k < CD_KMAX; k += blockDim.x) s_cnt[k] = 0;
    __syncthreads();
    int c = blockIdx.x * CD_CHUNK + threadIdx.x;
    if (c < nc) {
        int k = w.colour[c];
        if (k >= 0 && k < CD_KMAX) atomicAdd(&s_cnt[k], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < CD_KMAX; k += blockDim.x) w.chunk_cnt[k * ncl + blockIdx.x] = s_cnt[k];
}

template <int DIM, typename T>
__global__ void k_colour_scatter(CdGeom g, CdWork w, int pw)
{
    __shared__ int s_wcnt[CD_CHUNK / 32][CD_KMAX];
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int nc = ctrl->nc;
    const int ncl = live_chunks(nc);
    if ((int)blockIdx.x >= ncl) return;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (CD_CHUNK / 32) * CD_KMAX; i += blockDim.x) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    int c = blockIdx.x * CD_CHUNK + threadIdx.x;
    int k = (c < nc) ? w.colour[c] : -1;
    unsigned mask = __match_any_sync(0xffffffffu, k);
    int rank = __popc(mask & ((1u << lane) - 1u));
    if (k >= 0 && lane == __ffs(mask) - 1) s_wcnt[wid][k] = __popc(mask);
    __syncthreads();
    if (c >= nc || k < 0) return;
    for (int v = 0; v < wid; ++v) rank += s_wcnt[v][k];
    int pos = w.chunk_cnt[k * ncl + blockIdx.x] + rank;
    w.perm[pos] = c;
    int2 ab = w.pairs[c];
    w.c_ab[pos] = ab;
    double b = __ddiv_rn(w.gap[c], g.dt);
    if (DIM == 2) {
        typedef typename std::conditional<sizeof(T) == 8, double4_32a, float4>::type T4;
        typedef typename std::conditional<sizeof(T) == 8, double2, float2>::type T2;
        T4 geo;
        geo.x = (T)w.nrm[3 * c];
        geo.y = (T)w.nrm[3 * c + 1];
        geo.z = (T)b;
        geo.w = (T)w.mn[c];
        ((T4*)w.c_geo)[pos] = geo;
        ((T*)w.c_m)[pos] = (T)w.mt[c];
        T2 P;
        P.x = (T)w.Pk[2 * c];
        P.y = (T)w.Pk[2 * c + 1];
        ((T2*)w.c_P)[pos] = P;
    } else {
        typedef typename std::conditional<sizeof(T) == 8, double4_32a, float4>::type T4;
        typedef typename std::conditional<sizeof(T) == 8, double2, float2>::type T2;
        T4 geo;
        geo.x = (T)w.nrm[3 * c];
        geo.y = (T)w.nrm[3 * c + 1];
        geo.z = (T)w.nrm[3 * c + 2];
        geo.w = (T)b;
        ((T4*)w.c_geo)[pos] = geo;
        T2 m;
        m.x = (T)w.mn[c];
        m.y = (T)w.mt[c];
        ((T2*)w.c_m)[pos] = m;
        T4 P;
        P.x = (T)w.Pk[4 * c];
        P.y = (T)w.Pk[4 * c + 1];
        P.z = (T)w.Pk[4 * c + 2];
        P.w = (T)w.Pk[4 * c + 3];
        ((T4*)w.c_P)[pos] = P;
    }
}

__global__ void k_colour_offsets(CdWork w)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    int k = threadIdx.x;
    const int ncl = live_chunks(ctrl->nc);
    if (k < CD_KMAX) w.colour_off[k] = (ncl > 0) ? w.chunk_cnt[k * ncl] : 0;
    if (k == 0) w.colour_off[CD_KMAX] = ctrl->nc;
}

// Key-order contact range of each packing: contacts are sorted by body a and
// the packings' particles are consecutive, so packing b's contacts start at
// the first key whose a >= the packing's first particle.
__global__ void k_pk_ranges(CdGeom g, CdWork w)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    const int nc = ctrl->nc;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= g.npk; b += gridDim.x * blockDim.x) {
        if (b == g.npk) { w.pk_coff[b] = nc; continue; }
        const int first = w.pk[b].first;
        int lo = 0, hi = nc;
        while (lo < hi) {
            int mid = lo + ((hi - lo) >> 1);
            if (w.pairs[mid].x < first) lo = mid + 1; else hi = mid;
        }
        w.pk_coff[b] = lo;
    }
}

cudaError_t cd_launch_pk_ranges(const CdGeom& g, const CdWork& w, cudaStream_t s, int* nl)
{
    int gb = (g.npk + 1 + CD_BLOCK - 1) / CD_BLOCK;
    k_pk_ranges<<<gb, CD_BLOCK, 0, s>>>(g, w);
    ++*nl;
    return cudaGetLastError();
}

// Blocks per SM of the cooperative colouring grid (k_jp, and the merge's
// chain labelling, which runs on the same grid).  One keeps the grid barrier
// cheap: two made the 1e5-disc pile's colouring (29 rounds) 0.08 ms slower a
// step and the 1e6-sphere gas's (17 rounds) 0.02 ms faster.
#define CD_COLOUR_PER_SM 1

int cd_colour_max_blocks(int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jp, CD_SWEEP_THREADS, 0) != cudaSuccess) return 0;
    const int mg = cd_merge_label_blocks_per_sm();
    if (mg > 0 && mg < per_sm) per_sm = mg;
    if (per_sm > CD_COLOUR_PER_SM) per_sm = CD_COLOUR_PER_SM;
    return per_sm * num_sms;
}

cudaError_t cd_launch_colour(const CdGeom& g, const CdWork& w, int coop_blocks, int precision, int pw,
                             cudaStream_t s, int* nl, const double* pos)
{
    cudaError_t e;
    int nchunk = (g.cap + CD_CHUNK - 1) / CD_CHUNK;
    if (nchunk < 1) nchunk = 1;
    int gc = (g.cap + CD_BLOCK - 1) / CD_BLOCK;
    if (gc < 1) gc = 1;
    if (gc > 4096) gc = 4096;
    const int nbody = g.n + (g.dyn_walls ? 6 : 0);   // particles, then force-controlled walls n + k
    if ((e = cudaMemsetAsync(w.p2c_cnt, 0, sizeof(int) * (size_t)(nbody + 1), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.p2c_fill, 0, sizeof(int) * (size_t)nbody, s)) != cudaSuccess) return e;
    k_p2c_count<<<gc, CD_BLOCK, 0, s>>>(g, w); ++*nl;
    if ((e = cd_scan_exclusive(w.p2c_cnt, w.p2c_off, nbody + 1, w.scan_tmp, nullptr, s, nl)) != cudaSuccess) return e;
    k_p2c_fill<<<gc, CD_BLOCK, 0, s>>>(g, w); ++*nl;
    {
        int gn = (nbody + CD_BLOCK - 1) / CD_BLOCK;
        if (gn > 4096) gn = 4096;
        k_p2c_sort<<<gn, CD_BLOCK, 0, s>>>(g, w); ++*nl;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (coop_blocks > 0) {
        CdGeom ga = g;
        CdWork wa = w;
        unsigned long long* prio = w.prio;
        int* rc = w.round_cnt;
        void* args[] = {&ga, &wa, &prio, &rc};
        if ((e = cudaMemsetAsync(w.ctrl, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
        e = cudaLaunchCooperativeKernel((const void*)k_jp, dim3(coop_blocks), dim3(CD_SWEEP_THREADS), args, 0, s);
        if (e != cudaSuccess) return e;
        ++*nl;
    }
    if ((e = launch_repair(g, w, gc, s, nl)) != cudaSuccess) return e;
    k_chunk_hist<<<nchunk, CD_CHUNK, 0, s>>>(w); ++*nl;
    if ((e = cd_scan_exclusive(w.chunk_cnt, w.chunk_cnt, CD_KMAX * nchunk, w.scan_tmp, nullptr, s, nl,
                               &w.ctrl->chunk_last)) != cudaSuccess)
        return e;
    if (g.dim == 2) {
        if (precision == CD_FP64) k_colour_scatter<2, double><<<nchunk, CD_CHUNK, 0, s>>>(g, w, pw);
        else k_colour_scatter<2, float><<<nchunk, CD_CHUNK, 0, s>>>(g, w, pw);
        ++*nl;
    } else {
        if (precision == CD_FP64) k_colour_scatter<3, double><<<nchunk, CD_CHUNK, 0, s>>>(g, w, pw);
        else k_colour_scatter<3, float><<<nchunk, CD_CHUNK, 0, s>>>(g, w, pw);
        ++*nl;
    }
    k_colour_offsets<<<1, CD_KMAX, 0, s>>>(w); ++*nl;
    return cudaGetLastError();
}
