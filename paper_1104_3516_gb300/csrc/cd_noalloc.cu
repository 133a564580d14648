// cd_noalloc.cu -- contact detection for callers that cannot allocate device
// memory.
//
// Some hosts of this library run where cudaMalloc is not available to them:
// code inside a framework that owns every device allocation, a plug-in that
// may only use buffers handed to it, or a caller that must not allocate while
// a memory budget is fixed.  cd_detect_contacts_noalloc gives them the cell-
// list detection of cd_detect_contacts without a system object or workspace:
// its scratch (cell grid, per-particle counts and offsets, scan temporaries,
// pair mass matrix, a control block) lives in the file-scope device array
// below, which every GPU that loads the library holds until the process
// exits.
//
// The host cannot use the array's name as a device address, so on the first
// call on each device (with that device current) the address is looked up
// once with cudaGetSymbolAddress and cached; that first call therefore must
// not happen during stream capture.  All calls share the array and it keeps
// the last call's contents: every call clears what must start at zero, and
// calls that overlap on the GPU (two streams, two threads) race on it.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "cd_internal.cuh"

#define CD_NOALLOC_MAX_N 16384
#define CD_NOALLOC_MAX_CELLS 65536
#define CD_NOALLOC_MAX_CONTACTS 65536
#define CD_NOALLOC_MAX_DEVICES 64

// Byte layout of the scratch (each part 256-byte aligned).
#define NA_ALIGN(x) ((((size_t)(x)) + 255) & ~(size_t)255)
#define NA_CTRL 0
#define NA_I32(count) NA_ALIGN(sizeof(int) * (size_t)(count))
#define NA_CELL_OF (NA_CTRL + NA_ALIGN(sizeof(CdCtrl)))
#define NA_CELL_CNT (NA_CELL_OF + NA_I32(CD_NOALLOC_MAX_N))
#define NA_CELL_START (NA_CELL_CNT + NA_I32(CD_NOALLOC_MAX_CELLS + 1))
#define NA_CELL_FILL (NA_CELL_START + NA_I32(CD_NOALLOC_MAX_CELLS + 1))
#define NA_CELL_PID (NA_CELL_FILL + NA_I32(CD_NOALLOC_MAX_CELLS))
#define NA_PCNT (NA_CELL_PID + NA_I32(CD_NOALLOC_MAX_N))
#define NA_POFF (NA_PCNT + NA_I32(CD_NOALLOC_MAX_N + 1))
#define NA_SCAN (NA_POFF + NA_I32(CD_NOALLOC_MAX_N + 1))
#define NA_MN (NA_SCAN + NA_I32(CD_NOALLOC_MAX_CELLS / 1024 + 64))
#define NA_MT (NA_MN + NA_ALIGN(sizeof(double) * CD_NOALLOC_MAX_CONTACTS))
#define NA_PK (NA_MT + NA_ALIGN(sizeof(double) * CD_NOALLOC_MAX_CONTACTS))
#define NA_CAND (NA_PK + NA_ALIGN(sizeof(double) * 4 * CD_NOALLOC_MAX_CONTACTS))
#define NA_RMAX (NA_CAND + NA_I32((size_t)CD_NOALLOC_MAX_N * CD_CAND))
#define NA_BYTES (NA_RMAX + 256)

static __device__ __align__(256) unsigned char cd_noalloc_scratch[NA_BYTES];

static std::mutex na_mutex;
static void* na_addr[CD_NOALLOC_MAX_DEVICES];

// Largest radius (as ordered bits of a positive double) and a flag for any
// radius that is not positive and finite.
__global__ void k_noalloc_radii(int n, const double* __restrict__ radius, unsigned long long* out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double r = radius[i];
        if (!(r > 0.0) || !isfinite(r)) atomicMax(&out[1], 1ULL);
        else atomicMax(&out[0], (unsigned long long)__double_as_longlong(r));
    }
}

__global__ void k_noalloc_begin(CdCtrl* ctrl, unsigned long long* rmax_bits, double w0, double w1, double w2, double w3,
                                double w4, double w5)
{
    CdCtrl c;
    memset(&c, 0, sizeof c);
    c.wall_pos[0] = w0; c.wall_pos[1] = w1; c.wall_pos[2] = w2;
    c.wall_pos[3] = w3; c.wall_pos[4] = w4; c.wall_pos[5] = w5;
    *ctrl = c;
    rmax_bits[0] = 0ULL;
    rmax_bits[1] = 0ULL;
}

// Message of a failure, read back with cd_last_error(NULL).
void cd_set_global_error(const char* msg);

static cd_status na_error(cd_status st, const char* msg)
{
    cd_set_global_error(msg);
    return st;
}

static cd_status na_cuda(cudaError_t e, const char* where)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    cd_set_global_error(buf);
    return CD_ERR_CUDA;
}

extern "C" cd_status cd_detect_contacts_noalloc(const cd_params* params, int64_t n, const double* pos,
                                                const double* radius, const double* inv_mass,
                                                const double* inv_inertia, int64_t max_contacts, int32_t* pairs,
                                                double* normal, double* gap, int64_t* n_contacts, void* cuda_stream)
{
    cd_set_global_error("");
    if (!params || !pos || !radius || !inv_mass || !inv_inertia || !n_contacts)
        return na_error(CD_ERR_INVALID_ARG, "a required argument is NULL");
    const cd_params& p = *params;
    if (p.dim != 2 && p.dim != 3) return na_error(CD_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (n <= 0 || n > CD_NOALLOC_MAX_N)
        return na_error(CD_ERR_INVALID_ARG, "particle count must be in [1, 16384] for the no-allocation entry point");
    if (max_contacts < 0 || max_contacts > CD_NOALLOC_MAX_CONTACTS)
        return na_error(CD_ERR_INVALID_ARG, "max_contacts must be in [0, 65536] for the no-allocation entry point");
    if (max_contacts > 0 && (!pairs || !normal || !gap))
        return na_error(CD_ERR_INVALID_ARG, "pairs, normal and gap are required when max_contacts > 0");
    if (!(p.dt > 0.0) || !(p.delta >= 0.0)) return na_error(CD_ERR_INVALID_ARG, "dt must be > 0 and delta >= 0");
    for (int k = 0; k < p.dim; ++k)
        if (!(p.box_hi[k] > p.box_lo[k])) return na_error(CD_ERR_INVALID_ARG, "box_hi must exceed box_lo");
    for (int k = 0; k < 6; ++k)
        if (((p.wall_mask >> k) & 1) && ((k >> 1) >= p.dim || p.periodic[k >> 1]))
            return na_error(CD_ERR_INVALID_ARG, "wall on a missing or periodic axis");
    cudaStream_t s = (cudaStream_t)cuda_stream;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= CD_NOALLOC_MAX_DEVICES) return na_error(CD_ERR_INVALID_ARG, "device index out of range");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, cd_noalloc_scratch);
            if (e != cudaSuccess) return na_cuda(e, "cudaGetSymbolAddress");
            na_addr[dev] = ptr;
        }
        base = (unsigned char*)na_addr[dev];
    }

    CdCtrl* ctrl = (CdCtrl*)(base + NA_CTRL);
    unsigned long long* rbits = (unsigned long long*)(base + NA_RMAX);
    k_noalloc_begin<<<1, 1, 0, s>>>(ctrl, rbits, p.wall_pos[0], p.wall_pos[1], p.wall_pos[2], p.wall_pos[3],
                                    p.wall_pos[4], p.wall_pos[5]);
    int gb = (int)((n + CD_BLOCK - 1) / CD_BLOCK);
    k_noalloc_radii<<<gb, CD_BLOCK, 0, s>>>((int)n, radius, rbits);
    unsigned long long hb[2] = {0ULL, 0ULL};
    if ((e = cudaMemcpyAsync(hb, rbits, sizeof hb, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return na_cuda(e, "reading the largest radius");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return na_cuda(e, "cudaStreamSynchronize");
    if (hb[1]) return na_error(CD_ERR_INVALID_ARG, "radius must be positive and finite");
    double rmax;
    memcpy(&rmax, &hb[0], sizeof rmax);

    CdGeom g;
    memset(&g, 0, sizeof g);
    g.dim = (int)p.dim;
    g.n = (int)n;
    g.cap = (int)max_contacts;
    g.wall_mask = (int)p.wall_mask;
    g.delta = p.delta;
    g.dt = p.dt;
    g.mu = p.mu;
    g.rotations = (int)p.rotations;
    g.seed = p.seed;
    g.npk = 1;
    const double ell = (2.0 * rmax + p.delta) * (1.0 + 1e-9);   // as in cd_create_system
    long long ncell = 1;
    for (int k = 0; k < 3; ++k) {
        g.periodic[k] = (k < p.dim) ? (int)p.periodic[k] : 0;
        if (k < p.dim) {
            g.lo[k] = p.box_lo[k];
            g.hi[k] = p.box_hi[k];
            g.L[k] = p.box_hi[k] - p.box_lo[k];
            double m = std::floor(g.L[k] / ell);
            if (m < 1.0) m = 1.0;
            if (m > (double)CD_NOALLOC_MAX_CELLS) m = (double)CD_NOALLOC_MAX_CELLS;
            g.ncell[k] = (int)m;
            g.cs[k] = g.L[k] / m;
            g.inv_cs[k] = 1.0 / g.cs[k];
            if (g.periodic[k] && g.ncell[k] < 3)
                return na_error(CD_ERR_INVALID_ARG, "a periodic axis needs at least 3 cells (box >= 3 l)");
        } else {
            g.lo[k] = 0.0; g.hi[k] = 1.0; g.L[k] = 1.0; g.ncell[k] = 1; g.cs[k] = 1.0; g.inv_cs[k] = 1.0;
        }
        ncell *= g.ncell[k];
    }
    if (ncell > CD_NOALLOC_MAX_CELLS)
        return na_error(CD_ERR_INVALID_ARG, "the box needs more than 65536 cells for the no-allocation entry point");
    g.ncell_total = (int)ncell;

    CdWork w;
    memset(&w, 0, sizeof w);
    w.ctrl = ctrl;
    w.cell_of = (int*)(base + NA_CELL_OF);
    w.cell_cnt = (int*)(base + NA_CELL_CNT);
    w.cell_start = (int*)(base + NA_CELL_START);
    w.cell_fill = (int*)(base + NA_CELL_FILL);
    w.cell_pid = (int*)(base + NA_CELL_PID);
    w.pcnt = (int*)(base + NA_PCNT);
    w.poff = (int*)(base + NA_POFF);
    w.cand = (int*)(base + NA_CAND);
    w.scan_tmp = (int*)(base + NA_SCAN);
    w.mn = (double*)(base + NA_MN);
    w.mt = (double*)(base + NA_MT);
    w.Pk_nx = (double*)(base + NA_PK);
    w.Pk = w.Pk_nx;                 // the commit copy runs in place
    w.pairs_nx = (int2*)pairs;      // caller outputs
    w.pairs = (int2*)pairs;
    w.nrm = normal;
    w.gap = gap;
    w.pk_wall_pos = ctrl->wall_pos;   // device address inside the scratch
    const int pw = (p.dim == 2) ? 2 : 4;
    int nl = 0;
    if ((e = cd_launch_detect(g, w, pos, radius, inv_mass, inv_inertia, 0, pw, s, &nl)) != cudaSuccess)
        return na_cuda(e, "detection launch");
    CdCtrl h;
    if ((e = cudaMemcpyAsync(&h, ctrl, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return na_cuda(e, "reading the contact count");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return na_cuda(e, "cudaStreamSynchronize");
    *n_contacts = h.nc_needed;
    if (h.error == CDE_PER_PARTICLE) return na_error(CD_ERR_CAPACITY, "a particle has more than 64 contact candidates");
    if (h.overflow) return na_error(CD_ERR_CAPACITY, "more contacts than max_contacts; *n_contacts holds the number needed");
    return CD_OK;
}
