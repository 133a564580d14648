// cd_internal.cuh -- device-side layout and helpers shared by the CUDA
// translation units of the Contact Dynamics library (not a public header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cd_api.h"

#define CD_KMAX 64            // colours the ordering supports (bit mask in the colouring)
#define CD_MAXLOC 64          // pair candidates one particle may emit
#define CD_CAND 16            // partners the counting pass keeps per particle for the emitting pass
#define CD_SWEEP_THREADS 512  // threads per block of the persistent kernels
#define CD_BLOCK 256          // threads per block of the streaming kernels
#define CD_CHUNK 256          // contacts per chunk of the stable colour partition
#define CD_WAIT_NS 2000000000ULL  // bound on any device-side wait (2 s)
#define CD_MG_MAXC 3          // most colours one merged sweep phase takes
#define CD_MG_MIN_SWEEPS 64   // params.merge_last_colour 4: merge after solves of at least this many sweeps

// Device error codes written into CdCtrl::error.
enum { CDE_NONE = 0, CDE_TIMEOUT = 1, CDE_COLOURS = 2, CDE_PER_PARTICLE = 3, CDE_TAPE = 4 };

// Control block at the start of the workspace.
struct CdCtrl {
    unsigned long long bar_count;   // grid barrier: arrivals (monotone within a launch)
    unsigned long long bar_epoch;   // grid barrier: released epoch
    int nc;                         // contacts in the current set
    int nc_needed;                  // contacts found by the last detection
    int ncolours;
    int overflow;                   // 1: capacity exceeded in the current call
    int error;                      // CDE_* (timeouts, colour overflow)
    int skip;                       // 1: skip all remaining work of this call
    int uncoloured;
    int prev_offsets;               // 1: poff_prev holds the per-particle offsets of the current set
    long long sweeps;               // last solve
    long long converged;
    double residual;
    double r_avg;
    double wall_force[6];
    double wall_pos[6];             // moving wall planes
    // accumulated over the steps of one cd_step call
    long long steps_done;
    long long total_sweeps;
    long long total_updates;
    long long max_sweeps_step;
    long long n_not_conv;
    // last adjoint step
    long long adj_sweeps;
    long long adj_converged;
    double adj_residual;
    double adj_dmu;
    long long adj_nc;
    long long adj_nstick;
    long long adj_nslide;
    long long adj_nbodies;          // particles touched by a non-open contact
    long long adj_diverged;
    int tape_slot;                  // slot the next recorded step goes to
    int tape_pad;
    // merging of the last colours (params.merge_last_colour)
    int merge;                      // M > 0: this step's sweeps run the M last colours as one phase (-1: not this step)
    int mg_changed;                 // chain labelling: a label moved in the current round
    int mg_maxsize;                 // largest chain
    int mg_prev;                    // sweeps + 1 of the last solve (0: none yet), for params.merge_last_colour 4
    int chunk_last;                 // colour partition: CD_KMAX x live chunks - 1 (the scan's extent)
    int chunk_pad;
};

// Parameters of one packing of a batched system (a plain system is a batch of
// one).  Each packing has its own cell grid, walls, friction and gravity.
struct CdPack {
    double lo[3];
    double hi[3];
    double L[3];
    double cs[3];
    double inv_cs[3];               // 1 / cs (cell assignment)
    int ncell[3];
    int cell_base;      // first global cell id of this packing
    int periodic[3];
    int wall_mask;
    double mu;
    double gravity[3];
    double wall_vel[18];
    int first;          // first particle of the packing
    int count;          // particles of the packing
    unsigned long long seed;  // colouring seed of the packing
};

// Pointers into the caller's workspace.
struct CdWork {
    CdCtrl* ctrl;
    // particles
    void* V;            // packed velocity state (2D: 1 vec4, 3D: 2 vec4 per particle), real type
    void* S;            // packed static (inv_m, r, r/I, 0), real type
    int* cell_of;       // n
    int* cell_cnt;      // ncell + 1
    int* cell_start;    // ncell + 1
    int* cell_fill;     // ncell
    int* cell_pid;      // n
    int* pcnt;          // n + 1
    int* cand;          // n * CD_CAND: partners b > a found by the counting pass (first CD_CAND, found order)
    unsigned char* wmask; // n: walls in contact with each particle (bit k: wall k), from the counting pass (null: recomputed)
    float4* pf;         // n: (x, y, z, r) in single precision for the pair pre-filter (null: exact test only)
    int* poff;          // n + 1
    int* poff_prev;     // n + 1: poff of the current set (null: not kept)
    int* scan_tmp;      // block sums of the scans
    // contacts, key order
    int2* pairs;        // current set
    int2* pairs_nx;     // set being detected
    double* Pk;         // impulses of the current set (pw per contact)
    double* Pk_nx;
    double* nrm;        // 3 per contact
    double* gap;
    double* mn;
    double* mt;
    int* colour;
    // colouring
    int* p2c_cnt;       // n + 1
    int* p2c_off;       // n + 1
    int* p2c_fill;      // n
    int* p2c;           // 2 * cap
    unsigned long long* prio;  // cap colouring priorities
    int* round_cnt;     // 3 counters of the colouring rounds
    int* chunk_cnt;     // CD_KMAX * nchunk_cap + 1; used as [colour][live chunk]
    int* colour_off;    // CD_KMAX + 1
    int* perm;          // colour position -> key index
    // contacts, colour order (real type)
    int2* c_ab;
    void* c_geo;        // 2D: (nx, ny, b, mn)   3D: (nx, ny, nz, b)
    void* c_m;          // 2D: mt                3D: (mn, mt)
    void* c_P;          // 2D: (Pn, Pt)          3D: (Pn, Ptx, Pty, Ptz)
    double* partials;   // 2 * G * 4 reduction partials
    double* wpart;      // G * 6 wall-force partials
    // batched systems (npk packings)
    CdPack* pk;         // npk packing parameters
    int* pack_of;       // n: packing of each particle
    double* pk_wall_pos;// npk * 6 wall planes (aliases ctrl->wall_pos for one packing)
    int* pk_coff;       // npk + 1: key-order contact range of each packing
    int* pk_done;       // npk: 1 once the packing's convergence test passed
    double* pk_stats;   // npk * CD_PKSTATS per-packing statistics
    double* c_abs;      // cap (key order): |P| of the last update
    int* c_flag;        // cap (key order): local test bits of the last update
    int* act_cnt;       // 3 counters of packings still iterating, then 3 of their contacts
    // batched systems: second set of colour-order arrays for dropping the
    // contacts of converged packings during the solve
    int2* c_ab2;
    void* c_geo2;
    void* c_m2;
    void* c_P2;
    int* perm2;
    int* cmp_blk;       // G: kept contacts per block
    int* cmp_off;       // CD_KMAX + 1: colour offsets after dropping
    double* c_dpar;     // cap * pw (key order): impulse change of a parallel contact
    // domain-wise update (ndom_total > 1).  A particle whose contacts lie in
    // several domains has one velocity record per domain: its own record for
    // the lowest of them (its home), view records for the others (ascending
    // domain), each with the velocity of the sweep start beside it.
    int* dom_key;       // cap (key order): domain of each contact
    int* dom_home;      // n: lowest domain among the particle's contacts
    int* view_cnt;      // n + 1: view records of each particle
    int* view_off;      // n + 1: exclusive offsets; view_off[n] = views in use
    int* view_owner;    // 2 cap: particle of each view record
    void* V0;           // 2 cap velocity records: the sweep-start velocity of the view's particle
    int2* c_vab;        // cap (colour order): velocity records of bodies a and b
    // merging of the M last colours: their colour-order positions form chains
    // (contacts linked through a shared particle); chains are assigned whole
    // to the blocks of the sweep grid (arrays sized by capacity, used up to
    // the live contacts)
    int* mg_slot;       // CD_MG_MAXC x n: [m n + i] position of particle i's contact of colour K-M+m, or -1
    int* mg_label;      // cap: chain label (smallest position of the chain)
    int* mg_size;       // cap + 1: contacts of the chain labelled by the index
    int* mg_w;          // cap + 1: its contacts of colour K-M
    int* mg_start;      // cap + 1: exclusive scan of mg_w
    int* mg_bucket;     // cap: m G + block (colour K-M+m)
    int* mg_list;       // cap: positions grouped by bucket, ascending inside each
    int* mg_bcnt;       // CD_MG_MAXC G + 1: contacts per bucket
    int* mg_boff;       // CD_MG_MAXC G + 1: exclusive scan of mg_bcnt
    int* mg_bmin;       // CD_MG_MAXC G: lowest position of the bucket
    int* mg_bmax;       // CD_MG_MAXC G: highest position of the bucket
    // repair of the highest colour (global colour order)
    int* rep_top;       // npk: highest colour of each packing
    int* rep_dmax;      // npk: most contacts of one body of the packing
    int* rep_flag;      // cap + 1: 1 for a contact of its packing's highest colour
    int* rep_pos;       // cap + 1: exclusive scan of rep_flag
    int* rep_list;      // cap: those contacts in key order
    int* rep_path;      // cap: alternating path being followed (per packing: its contact range)
    double* obs;        // CD_OBS_MAX doubles: observable results
    // adjoint (params.tape_steps > 0)
    char* tape;         // tape_steps slots of CdTapeHdr + one step's records
    double2* adj_Y;     // cap: adjoint multipliers (Y_n, Y_t) of the contacts
    double4_16a* adj_B; // 2 n: per particle Gamma (x, y, w, 0) then Lambda (x, y, w, 0)
    double4_16a* adj_lam; // n: dL/dv of the step's velocities (x, y, w, 0)
    double2* adj_gx;    // n: dL/dx being accumulated
    int* adj_mark;      // n: 1 if the particle has a non-open contact
};

// One recorded time step for the adjoint (2D, FP64): the colour-order
// contact records after the solve and the velocities the step produced.
#define CD_GRAZING 1e-9   // P_n <= CD_GRAZING * max P_n: taken as open (touching, no force)
struct CdTapeHdr {
    int nc;
    int ncolours;
    int valid;          // 0 if the step was skipped or failed
    int pad;
    int colour_off[CD_KMAX + 1];
};
struct CdTape {
    CdTapeHdr* hdr;
    int2* ab;
    double4_16a* geo;   // nx, ny, b = g/dt, m_n
    double* mt;
    double2* P;         // converged (P_n, P_t)
    double4_16a* V;     // n: velocities after the step (vx, vy, w, 0)
};
__host__ __device__ inline size_t cd_align256(size_t x) { return (x + 255) & ~(size_t)255; }
__host__ __device__ inline size_t cd_tape_slot_bytes(int64_t n, int64_t cap)
{
    const size_t c = (size_t)(cap > 0 ? cap : 1), m = (size_t)(n > 0 ? n : 1);
    return cd_align256(sizeof(CdTapeHdr)) + cd_align256(c * sizeof(int2)) + cd_align256(c * sizeof(double4_16a)) +
           cd_align256(c * sizeof(double)) + cd_align256(c * sizeof(double2)) + cd_align256(m * sizeof(double4_16a));
}
__host__ __device__ inline CdTape cd_tape_slot(char* tape, int64_t n, int64_t cap, int slot)
{
    const size_t c = (size_t)(cap > 0 ? cap : 1);
    char* p = tape + (size_t)slot * cd_tape_slot_bytes(n, cap);
    CdTape t;
    t.hdr = (CdTapeHdr*)p;
    p += cd_align256(sizeof(CdTapeHdr));
    t.ab = (int2*)p;
    p += cd_align256(c * sizeof(int2));
    t.geo = (double4_16a*)p;
    p += cd_align256(c * sizeof(double4_16a));
    t.mt = (double*)p;
    p += cd_align256(c * sizeof(double));
    t.P = (double2*)p;
    p += cd_align256(c * sizeof(double2));
    t.V = (double4_16a*)p;
    return t;
}
#define CD_OBS_MAX 65536


// Per-packing statistics layout in pk_stats.
enum { PKS_SWEEPS = 0, PKS_CONV, PKS_RESID, PKS_RAVG, PKS_RPREV, PKS_NC, PKS_WF0, CD_PKSTATS = PKS_WF0 + 6 };

// Geometry of the problem in the form the kernels need.
struct CdGeom {
    int dim;
    int n;
    int cap;
    int periodic[3];
    int wall_mask;
    int ncell[3];
    double lo[3];
    double hi[3];
    double L[3];
    double cs[3];       // cell side per axis
    double inv_cs[3];   // 1 / cs (cell assignment)
    double delta;
    double dt;
    double mu;
    double gravity[3];
    double wall_vel[18];
    int rotations;
    int pad;
    unsigned long long seed;
    int npk;            // packings (1 for a plain system)
    int ncell_total;    // cells of all packings' grids
    double par_p;       // parallel fraction of the mixed update (0: Gauss-Seidel)
    int par_redraw;     // 1: the parallel subset is drawn afresh in every iteration step
    int dyn_walls;      // bit k: wall k is force-controlled (a body n + k in V, S, p2c)
    int pad2;
    double wall_im[6];  // inverse mass of a force-controlled wall, else 0
    double wall_push[6];// its push along the inward normal
    int ndom[3];        // domain-wise update (Sec. 3.1): slabs per axis (1: not cut)
    int ndom_total;     // product; > 1 selects the domain-wise sweep
    int merge_last;     // params.merge_last_colour (0 off, 2: at most two colours, 3: three, else two)
    int merge_auto;     // merge only after a solve of at least CD_MG_MIN_SWEEPS sweeps (or none yet)
    int merge_blocks;   // blocks of the sweep grid the chains are assigned to
};

// Velocity records of the domain views start after the particles' and the
// walls' records.
__host__ __device__ __forceinline__ int cd_view_base(const CdGeom& g) { return g.n + 6; }

// Body b takes part in conflicts and carries a velocity record: a particle or
// a force-controlled wall (plain systems).
__host__ __device__ __forceinline__ bool cd_is_body(const CdGeom& g, int b)
{
    return b < g.n || (g.dyn_walls != 0 && b - g.n < 6 && ((g.dyn_walls >> (b - g.n)) & 1));
}

// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea and Flood 2014) from its published definition; the
// colouring priority of contact key k is splitmix64(seed ^ k).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long cd_splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ unsigned long long cd_key(int a, int b)
{
    return ((unsigned long long)(unsigned)a << 32) | (unsigned long long)(unsigned)b;
}

// Mixed update (Sec. 2.3): a contact is in the parallel subset when a
// uniform number drawn for it (splitmix64 of its key mixed with the seed)
// falls below p.  sweep < 0: one fixed subset per contact key; sweep >= 0
// (params.parallel_redraw): the iteration step's number is mixed in as well,
// a fresh subset in every step.
__device__ __forceinline__ bool cd_is_parallel(double p, unsigned long long seed, unsigned long long key,
                                               long long sweep = -1)
{
    if (p <= 0.0) return false;
    if (p >= 1.0) return true;
    unsigned long long x = key ^ (seed * 0xD1B54A32D192ED03ULL);
    if (sweep >= 0) x ^= (unsigned long long)(sweep + 1) * 0x9E3779B97F4A7C15ULL;
    unsigned long long h = cd_splitmix64(x);
    double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    return u < p;
}

// ---------------------------------------------------------------------------
// Bounded grid barrier for cooperative launches (sense-reversing counter).
// Thread 0 of every block adds to one 32-bit word: block 0 adds
// 2^31 - (nblocks - 1), every other block adds 1, so the word's top bit flips
// exactly when the last block of the round arrives (all partial sums stay
// below 2^31 within a round) and the low bits return to their old value.
// Waiters compare the top bit with the value their own add returned.  The
// spin is bounded by %globaltimer (CD_WAIT_NS) and also stops early when
// another block has flagged an error; then it returns false (all threads of
// the block) and the caller must leave the kernel.  The word must be zero at
// launch (the launchers clear it).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long cd_globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned cd_ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int cd_ld_volatile_int(const int* p)
{
    return *(volatile const int*)p;
}

// Split form: cd_grid_arrive publishes the block's writes and adds its
// arrival (thread 0 gets the counter's old value); the block may then issue
// work that touches nothing another block reads before the barrier (loads of
// read-only records) while the others arrive; cd_grid_wait completes it.
__device__ __forceinline__ unsigned cd_grid_arrive(CdCtrl* ctrl, unsigned long long nblocks)
{
    __syncthreads();
    unsigned old = 0;
    if (threadIdx.x == 0) {
        unsigned* word = reinterpret_cast<unsigned*>(&ctrl->bar_count);
        const unsigned add = (blockIdx.x == 0) ? (0x80000000u - (unsigned)(nblocks - 1)) : 1u;
        // release: the block's writes (ordered before this thread by the block
        // barrier above) are visible to whoever acquires the flipped word
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(word), "r"(add) : "memory");
    }
    return old;
}

__device__ __forceinline__ bool cd_grid_wait(CdCtrl* ctrl, unsigned old, unsigned long long& epoch)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const unsigned* word = reinterpret_cast<const unsigned*>(&ctrl->bar_count);
        int ok = 1;
        unsigned long long t0 = 0;
        unsigned spins = 0;
        while (((cd_ld_acquire_u32(word) ^ old) & 0x80000000u) == 0u) {
            if ((++spins & 255u) == 0u) {
                if (t0 == 0) t0 = cd_globaltimer();
                else if (cd_globaltimer() - t0 > CD_WAIT_NS) {
                    atomicCAS(&ctrl->error, CDE_NONE, CDE_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (cd_ld_volatile_int(&ctrl->error) != CDE_NONE) { ok = 0; break; }
            }
        }
        // the acquire load that saw the flip orders thread 0's later accesses;
        // the block barrier below extends that to the other threads
        s_ok = ok;
        ++epoch;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool cd_grid_sync(CdCtrl* ctrl, unsigned long long nblocks, unsigned long long& epoch)
{
    const unsigned old = cd_grid_arrive(ctrl, nblocks);
    return cd_grid_wait(ctrl, old, epoch);
}

// ---------------------------------------------------------------------------
// The contacts [lo, hi) of one colour class spread evenly over the blocks of
// a persistent grid: block b takes the contiguous chunk b of ceil(count /
// blocks) positions and its threads stride over it.  (Handing out positions
// by global thread id would put a colour of 25k contacts on the first 49 of
// 152 SMs and make their FP64 pipes the bottleneck of every colour phase.)
// ---------------------------------------------------------------------------
struct CdSpan {
    int p;      // this thread's first position
    int end;    // end of the block's chunk
};
__device__ __forceinline__ CdSpan cd_colour_span(int lo, int hi)
{
    const int cnt = hi - lo;
    const int chunk = (cnt + (int)gridDim.x - 1) / (int)gridDim.x;
    const int b0 = lo + (int)blockIdx.x * chunk;
    CdSpan s;
    s.p = b0 + (int)threadIdx.x;
    s.end = (b0 + chunk < hi) ? b0 + chunk : hi;
    return s;
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files), all on `stream`.
// ---------------------------------------------------------------------------
cudaError_t cd_scan_exclusive(const int* in, int* out, int n, int* tmp, int* total_dst, cudaStream_t stream,
                              int* nl, const int* n_dev = nullptr);
size_t cd_scan_tmp_ints(int n);

cudaError_t cd_launch_detect(const CdGeom& g, const CdWork& w, const double* pos, const double* radius,
                             const double* inv_m, const double* inv_I, int warm, int pw, cudaStream_t stream, int* nl);
cudaError_t cd_launch_set_contacts(const CdGeom& g, const CdWork& w, const double* pos, const double* radius,
                                   const double* inv_m, const double* inv_I, int nc, const int32_t* pairs,
                                   const double* impulses, int pw, cudaStream_t stream, int* nl);
cudaError_t cd_launch_colour(const CdGeom& g, const CdWork& w, int coop_blocks, int precision, int pw,
                             cudaStream_t stream, int* nl, const double* pos);
cudaError_t cd_launch_pack(const CdGeom& g, const CdWork& w, const double* vel, const double* omega,
                           const double* radius, const double* inv_m, const double* inv_I, const double* f_ext,
                           int free_flight, int precision, cudaStream_t stream, int* nl);
cudaError_t cd_launch_domains(const CdGeom& g, const CdWork& w, const double* pos, const double* radius,
                              cudaStream_t stream, int* nl);
cudaError_t cd_launch_merge(const CdGeom& g, const CdWork& w, int coop_blocks, cudaStream_t stream, int* nl);
int cd_merge_label_blocks_per_sm();
cudaError_t cd_launch_pk_ranges(const CdGeom& g, const CdWork& w, cudaStream_t stream, int* nl);
cudaError_t cd_launch_orient(const CdGeom& g, const CdWork& w, int nbins, unsigned long long* counts,
                             cudaStream_t stream, int* nl);
// Records the step just taken into slot ctrl->tape_slot of the tape (T slots)
// and advances the slot, all on the device (so a captured step graph can be
// replayed).
cudaError_t cd_launch_tape_record(const CdGeom& g, const CdWork& w, int64_t cap, int T, cudaStream_t stream, int* nl);
cudaError_t cd_launch_set_tape_slot(const CdWork& w, int slot, cudaStream_t stream, int* nl);
struct CdAdjIO {
    const double* dLx;      // n*2: dL/dx' of the step's output positions
    const double* dLv;      // n*2: dL/dv'
    const double* dLw;      // n:   dL/domega'
    double* ox;             // n*2: dL/dx of the step's input positions
    double* ov;             // n*2: dL/dv
    double* ow;             // n:   dL/domega
    const double* inv_I;    // n
    double wq[6];           // dL/d(wall force k) / dt: weight of the normal impulse of a contact with wall k
    double eps;             // relative compliance of the rows (params.adjoint_compliance)
};
cudaError_t cd_launch_adjoint(const CdGeom& g, const CdWork& w, const CdTape& t, const CdAdjIO& io, double alpha,
                              int max_sweeps, int coop_blocks, cudaStream_t stream, int* nl);
int cd_adjoint_blocks_per_sm();
cudaError_t cd_launch_stress(const CdGeom& g, const CdWork& w, const double* pos, const double* radius, int axis,
                             double lo, double width, int ns, double* sig, cudaStream_t stream, int* nl);
cudaError_t cd_launch_sweep(const CdGeom& g, const CdWork& w, int coop_blocks, int threads, int precision,
                            int criterion, double alpha, int max_sweeps, int pw, cudaStream_t stream, int* nl);
int cd_sweep_fits(const CdGeom& g, int precision, int threads, int per_sm);
cudaError_t cd_launch_unpack(const CdGeom& g, const CdWork& w, double* pos, double* vel, double* omega,
                             double* theta, int integrate, int precision, cudaStream_t stream, int* nl);
cudaError_t cd_launch_static(const CdGeom& g, const CdWork& w, const double* radius, const double* inv_m,
                             const double* inv_I, int precision, cudaStream_t stream, int* nl);
int cd_sweep_max_blocks(int precision, int dim, int num_sms);
int cd_colour_max_blocks(int num_sms);
