// cd_sweep.cu -- the iterative contact-impulse solve (paper Sec. 2.1, Fig. 2)
// and the Euler update (Eqs. 1-2).
//
// k_sweep is one cooperative persistent launch per solve: it applies the
// starting impulses, then repeats sweeps over the colour classes (one grid
// barrier per colour) until the convergence test of Sec. 2.1 passes or the
// sweep cap is hit.  All blocks compute the residual from the same per-block
// partial sums in the same order, so they agree on when to stop without any
// host round trip.
//
// Single-contact update (Fig. 2), in impulses P = R dt.  With u the current
// relative velocity of the contact points (this contact's own impulse
// included) and M = diag(m_n, m_t) the pair mass matrix (Eq. 5), removing the
// own impulse gives v_g0 = u - M^-1 P_old, so the sticking impulse of Eq. 5,
// P = -M (g/dt n + v_g0), reads
//     P_n* = P_n,old - m_n (g/dt + u_n),   P_t* = P_t,old - m_t u_t.
// Eq. 3 (gap stays open) is P_n* < 0 -> P = 0; the Coulomb test (Eq. 8) and
// the sliding solution (Eqs. 9-11: tangential impulse of magnitude mu P_n
// against the sliding velocity, which for discs and spheres is parallel to
// P_t*) give P_t = P_t* scaled onto |P_t| <= mu P_n.
#include <type_traits>

#include "cd_internal.cuh"

// Variants of the persistent colour-barrier sweep: plain Gauss-Seidel, the
// mixed update of Sec. 2.3, the domain-wise update of Sec. 3.1.
enum { CD_SWEEP_PLAIN = 0, CD_SWEEP_MIXED = 1, CD_SWEEP_DOMAINS = 2, CD_SWEEP_MERGE = 3 };

// Merged last phase of a step (params.merge_last_colour): phase `klast` runs
// the M last colours in place of M phases.  This block's positions of colour
// K-M+m are mg_list[lst[2m] .. lst[2m + 1]) (lst in shared memory).  The
// block's items are numbered through the M lists in turn;
// item q goes to thread q % blockDim, so a thread's first item (prefetched
// before the grid barrier) may belong to any of the lists, and the later
// sub-steps wait after their block barrier only for their velocities.
struct MgInfo {
    int on;
    int klast;
    int M;
    const int* lst;
    long long draw;   // mixed update: the iteration step whose parallel subset applies (-1: fixed subset)
};

template <typename T> struct Vec;
// FP64 records are 32 bytes at 32-byte aligned addresses (every workspace array
// is 256-byte aligned): one 256-bit access per record
template <> struct Vec<double> { typedef double4_32a V4; typedef double2 V2; };
template <> struct Vec<float> { typedef float4 V4; typedef float2 V2; };

// Arithmetic of the sweep's real type with the rounding written out (no
// contraction left to the compiler): fused multiply-add rounded once,
// product, sum and difference.
template <typename T> __device__ __forceinline__ T fma_of(T a, T b, T c);
template <> __device__ __forceinline__ double fma_of<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <> __device__ __forceinline__ float fma_of<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <typename T> __device__ __forceinline__ T mul_of(T a, T b);
template <> __device__ __forceinline__ double mul_of<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float mul_of<float>(float a, float b) { return __fmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T add_of(T a, T b);
template <> __device__ __forceinline__ double add_of<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float add_of<float>(float a, float b) { return __fadd_rn(a, b); }
template <typename T> __device__ __forceinline__ T sub_of(T a, T b);
template <> __device__ __forceinline__ double sub_of<double>(double a, double b) { return __dsub_rn(a, b); }
template <> __device__ __forceinline__ float sub_of<float>(float a, float b) { return __fsub_rn(a, b); }

// Stores the first three components of a velocity record, leaving the fourth.
template <typename T>
__device__ __forceinline__ void store_xyz_plain(typename Vec<T>::V4* dst, const typename Vec<T>::V4& v)
{
    typedef typename Vec<T>::V2 T2;
    T2 xy;
    xy.x = v.x; xy.y = v.y;
    *reinterpret_cast<T2*>(dst) = xy;
    reinterpret_cast<T*>(dst)[2] = v.z;
}

// ---------------------------------------------------------------------------
// Static per-particle record (inv_m, r, r / I, 0) in the sweep's real type.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_static(CdGeom g, int n, int rotations, const double* __restrict__ radius,
                         const double* __restrict__ inv_m, const double* __restrict__ inv_I,
                         typename Vec<T>::V4* __restrict__ S)
{
    // records n .. n + 5: force-controlled walls (inverse mass, no radius, no rotation)
    if (blockIdx.x == 0 && threadIdx.x < 6) {
        typename Vec<T>::V4 s;
        s.x = (T)(((g.dyn_walls >> threadIdx.x) & 1) ? g.wall_im[threadIdx.x] : 0.0);
        s.y = (T)0; s.z = (T)0; s.w = (T)0;
        S[n + threadIdx.x] = s;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        typename Vec<T>::V4 s;
        double r = radius[i];
        s.x = (T)inv_m[i];
        s.y = (T)r;
        s.z = rotations ? (T)(r * inv_I[i]) : (T)0;
        s.w = (T)0;
        S[i] = s;
    }
}

// ---------------------------------------------------------------------------
// Packs the caller's velocities into the sweep state; with free_flight the
// explicit external forces of Eq. 1 are applied first (F = m g + f_ext).
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void k_pack(CdGeom g, CdWork w, const double* __restrict__ vel, const double* __restrict__ omega,
                       const double* __restrict__ inv_m, const double* __restrict__ f_ext, int free_flight)
{
    if (w.ctrl->skip) return;
    typedef typename Vec<T>::V4 T4;
    T4* V = (T4*)w.V;
    // force-controlled walls: velocity records n + k, pushed along the inward normal (Eq. 1)
    if (g.dyn_walls && blockIdx.x == 0 && threadIdx.x < 6 && ((g.dyn_walls >> threadIdx.x) & 1)) {
        const int k = threadIdx.x, ax = k >> 1;
        double u[3] = {w.pk[0].wall_vel[3 * k], w.pk[0].wall_vel[3 * k + 1], w.pk[0].wall_vel[3 * k + 2]};
        if (free_flight) {
            double a = __dmul_rn(g.wall_push[k], g.wall_im[k]);
            if (k & 1) a = -a;
            u[ax] = __dadd_rn(u[ax], __dmul_rn(a, g.dt));
        }
        T4 s;
        s.x = (T)u[0]; s.y = (T)u[1]; s.z = (T)((DIM == 3) ? u[2] : 0.0); s.w = (T)0;
        if (DIM == 2) {
            V[g.n + k] = s;
        } else {
            T4 o;
            o.x = (T)0; o.y = (T)0; o.z = (T)0; o.w = (T)0;
            V[2 * (g.n + k)] = s;
            V[2 * (g.n + k) + 1] = o;
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        double v[3] = {0.0, 0.0, 0.0};
        double im = inv_m[i];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            double vk = vel[i * DIM + k];
            if (free_flight) {
                double gk = (g.npk > 1) ? w.pk[w.pack_of[i]].gravity[k] : g.gravity[k];
                double a = (im == 0.0) ? 0.0 : gk;
                if (f_ext) a = __dadd_rn(a, __dmul_rn(f_ext[i * DIM + k], im));
                vk = __dadd_rn(vk, __dmul_rn(a, g.dt));
            }
            v[k] = vk;
        }
        if (DIM == 2) {
            T4 s;
            s.x = (T)v[0]; s.y = (T)v[1]; s.z = (T)omega[i]; s.w = (T)0;
            V[i] = s;
        } else {
            T4 s, o;
            s.x = (T)v[0]; s.y = (T)v[1]; s.z = (T)v[2]; s.w = (T)0;
            o.x = (T)omega[3 * i]; o.y = (T)omega[3 * i + 1]; o.z = (T)omega[3 * i + 2]; o.w = (T)0;
            V[2 * i] = s;
            V[2 * i + 1] = o;
        }
    }
}

// ---------------------------------------------------------------------------
// Unpacks the sweep state into the caller's velocities; with integrate the
// positions (and 2D orientations) follow Eq. 2 and the walls move.
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void k_unpack(CdGeom g, CdWork w, double* __restrict__ pos, double* __restrict__ vel,
                         double* __restrict__ omega, double* __restrict__ theta, int integrate)
{
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    typedef typename Vec<T>::V4 T4;
    const T4* V = (const T4*)w.V;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        double v[3], om[3];
        if (DIM == 2) {
            T4 s = V[i];
            v[0] = (double)s.x; v[1] = (double)s.y; v[2] = 0.0;
            om[0] = (double)s.z;
        } else {
            T4 s = V[2 * i], o = V[2 * i + 1];
            v[0] = (double)s.x; v[1] = (double)s.y; v[2] = (double)s.z;
            om[0] = (double)o.x; om[1] = (double)o.y; om[2] = (double)o.z;
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            vel[i * DIM + k] = v[k];
            if (integrate) {
                double xn = __dadd_rn(pos[i * DIM + k], __dmul_rn(v[k], g.dt));
                if (g.periodic[k]) {
                    if (xn >= g.hi[k]) xn = __dsub_rn(xn, g.L[k]);
                    else if (xn < g.lo[k]) xn = __dadd_rn(xn, g.L[k]);
                }
                pos[i * DIM + k] = xn;
            }
        }
        if (DIM == 2) {
            omega[i] = om[0];
            if (integrate && theta) theta[i] = __dadd_rn(theta[i], __dmul_rn(om[0], g.dt));
        } else {
            omega[3 * i] = om[0]; omega[3 * i + 1] = om[1]; omega[3 * i + 2] = om[2];
        }
    }
    if (g.dyn_walls && blockIdx.x == 0 && threadIdx.x == 0) {
        // force-controlled walls: their velocity after the solve becomes the wall velocity
        for (int k = 0; k < 2 * DIM; ++k) {
            if (!((g.dyn_walls >> k) & 1)) continue;
            const T4 s = (DIM == 2) ? V[g.n + k] : V[2 * (g.n + k)];
            const double u[3] = {(double)s.x, (double)s.y, (double)s.z};
            w.pk[0].wall_vel[3 * k + (k >> 1)] = u[k >> 1];
        }
    }
    if (integrate) {
        if (g.dyn_walls) __syncthreads();   // block 0 moves the walls after their velocities are written
        for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < g.npk; b += gridDim.x * blockDim.x) {
            const CdPack& pb = w.pk[b];
            for (int k = 0; k < 2 * DIM; ++k)
                if ((pb.wall_mask >> k) & 1)
                    w.pk_wall_pos[6 * b + k] = __dadd_rn(w.pk_wall_pos[6 * b + k],
                                                         __dmul_rn(pb.wall_vel[3 * k + (k >> 1)], g.dt));
        }
    }
}

// ---------------------------------------------------------------------------
// Deterministic reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the warp, or +0 without any FP64 instruction when every lane
// holds +0 (a warp of idle threads: the narrow FP64 pipe would spend the
// same time on it as on a busy warp).  The same bits as warp_sum.
__device__ __forceinline__ double warp_sum_nz(double v)
{
    if (!__any_sync(0xffffffffu, __double_as_longlong(v) != 0)) return v;
    return warp_sum(v);
}

// Block sum of the first nv of NV values per thread (fixed tree); result
// valid in thread 0.  Values nv .. NV-1 stay the thread's own (callers pass
// nv < NV only when those values are zero everywhere).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*s_red)[NV], int nv = NV)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j)
        if (j < nv) v[j] = warp_sum_nz(v[j]);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j < nv) s_red[wid][j] = v[j];
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            if (j < nv) {
                double x = (lane < nw) ? s_red[lane][j] : 0.0;
                v[j] = warp_sum_nz(x);
            }
        }
    }
    __syncthreads();
}

// Sum over blocks of partial field f, identical in every block: lanes of warp
// 0 stride over the blocks in order, then a fixed butterfly; broadcast.
__device__ __forceinline__ double grid_total(const double* part, int nblocks, double* s_bcast)
{
    if (threadIdx.x < 32) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 32) x += part[b];
        x = warp_sum(x);
        if (threadIdx.x == 0) *s_bcast = x;
    }
    __syncthreads();
    double r = *s_bcast;
    __syncthreads();
    return r;
}

// Values of the per-block partials a sweep's convergence test reads (the
// counts of test II only under that test).
__device__ __forceinline__ int test_values(int crit) { return crit == CD_CONV_LOCAL ? 3 : 1; }

// The convergence test after a sweep (tests I and II) from the block
// partials part[0 .. 3 nb): the block's last warp sums them (the order of
// grid_total) and its lane 0 decides; the result reaches the block through
// shared memory (s_b3, three doubles), so the FP64 divisions run once per
// block.  The last warp holds the fewest contacts of a colour phase (they
// are dealt from thread 0 up), so the other warps' work before the block
// barrier below (the next sweep's first updates, staged) overlaps the test.
__device__ __forceinline__ void sweep_test(const double* part, int nb, int nc, int crit, double alpha,
                                           double ravg_prev, double& ravg, double& resid, int& converged,
                                           double* s_b3)
{
    if ((threadIdx.x >> 5) == (blockDim.x >> 5) - 1) {
        const int lane = threadIdx.x & 31;
        const bool local = (crit == CD_CONV_LOCAL);
        double x = 0.0, xr = 0.0, xb = 0.0;
        for (int b = lane; b < nb; b += 32) {
            x += part[b];
            if (local) { xr += part[nb + b]; xb += part[2 * nb + b]; }
        }
        x = warp_sum(x);
        if (local) { xr = warp_sum(xr); xb = warp_sum(xb); }
        if (lane == 0) {
            const double ra = x / (double)nc;
            const double den = ra + ravg_prev;
            double rs;
            int cv;
            if (crit == CD_CONV_GLOBAL_REL) {
                rs = (den > 0.0) ? fabs(ra - ravg_prev) / den : (den == 0.0 ? 0.0 : den);
                cv = rs < alpha;
            } else if (crit == CD_CONV_GLOBAL_SQ) {
                double q = (den > 0.0) ? (ra - ravg_prev) / den : (den == 0.0 ? 0.0 : den);
                rs = q * q;
                cv = rs < alpha;
            } else if (local) {
                rs = (double)(nc - (long long)xr) / (double)nc;
                cv = (10.0 * xr >= 9.0 * (double)nc) && xb == 0.0;
            } else {
                rs = (den > 0.0) ? fabs(ra - ravg_prev) / den : (den == 0.0 ? 0.0 : den);
                cv = 0;
            }
            s_b3[0] = ra;
            s_b3[1] = rs;
            s_b3[2] = (double)cv;
        }
    }
    __syncthreads();
    ravg = s_b3[0];
    resid = s_b3[1];
    converged = (s_b3[2] != 0.0);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Single-contact updates (Fig. 2).  A contact record holds everything of the
// update except the two bodies' velocities: it is read-only within a colour
// phase, so a thread loads its next record before the grid barrier and only
// the velocity loads sit on the critical path after it.
// ---------------------------------------------------------------------------
struct UpdOut {
    double pabs;     // |P| after the update (deferred form: |P| of the thread's previous update)
    double psq;      // |P|^2 after the update (3D and FP32)
    double pn, pt;   // deferred form (FP64 2D): P_n, P_t after the update
    int rel_ok;      // local test (I), relative branch
    int bad;         // local test (I): fails both branches
};

template <int DIM, typename T> struct Rec;
template <typename T> struct Rec<2, T> {
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    T mu;        // friction coefficient of the contact's packing
    int pk;      // packing of body a
    int2 ab;
    T4 geo;      // nx, ny, b = g/dt, m_n
    T mt;
    T2 P;        // P_n, P_t before the update
    T4 sa, sb;   // inv_m, r, r/I, 0 (sb = 0 for a wall)
    int2 vab;    // domain-wise update only: velocity records of a and b
};
template <typename T> struct Rec<3, T> {
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    T mu;
    int pk;
    int2 ab;
    T4 geo;      // nx, ny, nz, b = g/dt
    T2 m;        // m_n, m_t
    T4 P;        // P_n, P_tx, P_ty, P_tz before the update
    T4 sa, sb;
    int2 vab;
};

// The bodies' static records (inv_m, r, r/I).  FP64: loaded with the
// velocities, after the barrier, not with the prefetched record (their
// loads run in parallel with the velocity loads, and the record held across
// the barrier stays 16 registers smaller: no spills at the 128-register
// cap; 2D sweep 28.56 -> 28.28 ms per step).  FP32 (no spills, 16-byte
// records): with the prefetched record, which was 2% faster there.
template <int DIM, typename T>
__device__ __forceinline__ void load_static(const CdGeom& g, const CdWork& w, Rec<DIM, T>& r)
{
    typedef typename Vec<T>::V4 T4;
    const T4* S = (const T4*)w.S;
    r.sa = S[r.ab.x];
    if (cd_is_body(g, r.ab.y)) {   // a particle, or a force-controlled wall (record n + k)
        r.sb = S[r.ab.y];
    } else {
        r.sb.x = (T)0; r.sb.y = (T)0; r.sb.z = (T)0; r.sb.w = (T)0;
    }
}

// VIEWS: the domain-wise update, whose contacts work on their domain's
// velocity records (c_vab); otherwise the records are the bodies' own.
template <int DIM, typename T, bool VIEWS = false>
__device__ __forceinline__ void load_rec(const CdGeom& g, const CdWork& w, int pos, Rec<DIM, T>& r)
{
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    r.ab = w.c_ab[pos];
    if (g.npk > 1) {
        r.pk = w.pack_of[r.ab.x];
        r.mu = (T)w.pk[r.pk].mu;
    } else {
        r.pk = 0;
        r.mu = (T)g.mu;
    }
    r.geo = ((const T4*)w.c_geo)[pos];
    if constexpr (DIM == 2) {
        r.mt = ((const T*)w.c_m)[pos];
        r.P = ((const T2*)w.c_P)[pos];
    } else {
        r.m = ((const T2*)w.c_m)[pos];
        r.P = ((const T4*)w.c_P)[pos];
    }
    if constexpr (sizeof(T) == 4) load_static<DIM, T>(g, w, r);
    if constexpr (VIEWS) r.vab = w.c_vab[pos];
}



// max(x, 0) and the projection of x onto [-lim, lim] (lim >= 0).  For FP64
// they are done on the bit patterns with integer instructions (non-negative
// doubles order like their 64-bit integer images), which keeps them off the
// narrow FP64 pipe; the results are exactly those of the comparisons.
__device__ __forceinline__ double pos_part(double x)
{
    long long b = __double_as_longlong(x);
    return b < 0 ? 0.0 : x;
}
__device__ __forceinline__ float pos_part(float x) { return x > 0.0f ? x : 0.0f; }

__device__ __forceinline__ double clamp_sym(double x, double lim)
{
    unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    unsigned long long bl = (unsigned long long)__double_as_longlong(lim);
    unsigned long long ax = bx & 0x7FFFFFFFFFFFFFFFULL;
    return ax > bl ? __longlong_as_double((long long)(bl | (bx & 0x8000000000000000ULL))) : x;
}
__device__ __forceinline__ float clamp_sym(float x, float lim) { return x < -lim ? -lim : (x > lim ? lim : x); }

// |P| = sqrt(s) from |P|^2 for the residual only, in two FP64 instructions
// (the FP64 pipe is the narrow one).  Write s = m 4^k with m in [1, 4) by
// exponent arithmetic on the bit pattern; take the FP32 reciprocal square
// root z of m rounded to FP32 (correctly rounded, __frsqrt_rn) and the FP32
// product y = m z, both on the wide FP32 pipe and widened exactly; then one
// Newton step of Heron's iteration for sqrt(m) from y, with z / 2 for
// 1 / (2 y): y + (m - y^2) z / 2; scale by 2^k.  With y = sqrt(m) (1 + d),
// |d| <= 2.5 2^-24 (three FP32 roundings), and z sqrt(m) = 1 + e, |e| <=
// 1.5 2^-24, the result is sqrt(m) (1 - d^2 / 2 - d e + O(d^3)): within
// 2.5e-14 relative.  Subnormal and infinite s take
// s * rsqrt(s); zero and negative s give 0; a NaN with the sign bit clear
// (what arithmetic on NaN produces here) gives NaN, as sqrt would, so that a
// diverged iteration does not look converged to the residual test; the
// decision is on the bit pattern, with no FP64 compare.
__device__ __forceinline__ double norm_of_sq(double s)
{
    const long long b = __double_as_longlong(s);
    const int be = (int)(b >> 52);   // biased exponent (sign clear for s >= 0)
    if (be <= 0 || be >= 0x7FF)
        return (b > 0 && b <= 0x7FF0000000000000LL) ? s * rsqrt(s) : (b > 0x7FF0000000000000LL ? s : 0.0);
    const int e = be - 1023;
    const int k = e >> 1;   // floor(e / 2)
    const long long mb = (b & 0x000FFFFFFFFFFFFFLL) | ((long long)(1023 + e - 2 * k) << 52);
    const double m = __longlong_as_double(mb);
    // m to FP32, rounded to nearest (a carry into the exponent is the rounding)
    const float mf = __int_as_float((int)(((mb + (1LL << 28)) >> 29) - (896LL << 23)));
    const float zf = __frsqrt_rn(mf);   // in [0.5, 1]
    const long long zb = ((long long)__float_as_int(zf) << 29) + (896LL << 52);   // exact widening
    const double h = __longlong_as_double(zb - (1LL << 52));                      // z / 2
    const float yf = __fmul_rn(mf, zf);                                            // ~sqrt(m), in (0.9, 2.1)
    const double y = __longlong_as_double(((long long)__float_as_int(yf) << 29) + (896LL << 52));   // exact
    const double r = __fma_rn(-y, y, m);
    const double y1 = __fma_rn(r, h, y);
    return __longlong_as_double(__double_as_longlong(y1) + ((long long)k << 52));
}

// |P| from the |P|^2 an update left (in the sweep's real type: FP32 impulses
// carry 1e-7 anyway, their magnitude is taken in FP32).  The persistent FP64
// 2D sweep defers it: a thread takes the magnitude of its previous update
// while the velocity loads of its next one are in flight, when the narrow
// FP64 pipe has nothing else to do; the per-thread sum sees the same terms in
// the same order, so the residual is bit-identical.
template <typename T> __device__ __forceinline__ double abs_of_sq(double s);
template <> __device__ __forceinline__ double abs_of_sq<double>(double s) { return norm_of_sq(s); }
template <> __device__ __forceinline__ double abs_of_sq<float>(double s) { return (double)sqrtf((float)s); }

// |P|^2 = P_n^2 + P_t^2 with a fixed rounding (the FP64 2D sweeps take it
// either inline or deferred, and must agree), and |P| from the pair.
__device__ __forceinline__ double sq2(double a, double b) { return __fma_rn(b, b, __dmul_rn(a, a)); }
__device__ __forceinline__ double abs_of_pair(double pn, double pt) { return norm_of_sq(sq2(pn, pt)); }

// 2D: P_n = max(0, P_n,old - m_n (b + u_n)); P_t = clamp(P_t,old - m_t u_t, +-mu P_n).
template <typename T, bool SQ = false>
__device__ __forceinline__ UpdOut core2d(const CdGeom& g, const Rec<2, T>& r, typename Vec<T>::V4& va,
                                         typename Vec<T>::V4& vb, bool wall, bool apply_only, int crit,
                                         double alpha, double ravg_prev, typename Vec<T>::V2& Pnew)
{
    // every operation is written out (fused steps where they save an
    // instruction): each kernel and call site that inlines this computes the
    // same bits
    const T nx = r.geo.x, ny = r.geo.y;
    T Pn, Pt, dPn, dPt;
    if (apply_only) {
        Pn = r.P.x; Pt = r.P.y;
        dPn = Pn; dPt = Pt;
    } else {
        const T b = r.geo.z, mn = r.geo.w;
        const T dvx = sub_of<T>(vb.x, va.x), dvy = sub_of<T>(vb.y, va.y);
        const T un = fma_of<T>(dvy, ny, mul_of<T>(dvx, nx));
        // u_t = (dv x n) - (r_a w_a + r_b w_b)
        T ut = fma_of<T>(dvy, nx, -mul_of<T>(dvx, ny));
        ut = fma_of<T>(-r.sa.y, va.z, ut);
        ut = fma_of<T>(-r.sb.y, vb.z, ut);
        Pn = pos_part(fma_of<T>(-mn, add_of<T>(b, un), r.P.x));
        const T lim = mul_of<T>(r.mu, Pn);
        Pt = clamp_sym(fma_of<T>(-r.mt, ut, r.P.y), lim);
        dPn = sub_of<T>(Pn, r.P.x);
        dPt = sub_of<T>(Pt, r.P.y);
    }
    const T dPx = fma_of<T>(dPn, nx, -mul_of<T>(dPt, ny));
    const T dPy = fma_of<T>(dPn, ny, mul_of<T>(dPt, nx));
    va.x = fma_of<T>(-r.sa.x, dPx, va.x);
    va.y = fma_of<T>(-r.sa.x, dPy, va.y);
    va.z = fma_of<T>(-r.sa.z, dPt, va.z);
    if (!wall) {
        vb.x = fma_of<T>(r.sb.x, dPx, vb.x);
        vb.y = fma_of<T>(r.sb.x, dPy, vb.y);
        vb.z = fma_of<T>(-r.sb.z, dPt, vb.z);
    }
    Pnew.x = Pn; Pnew.y = Pt;
    UpdOut o;
    const double pn = (double)Pn, pt = (double)Pt;
    // SQ (FP64): the pair only, the magnitude is taken later (abs_of_pair)
    o.pn = pn;
    o.pt = pt;
    if constexpr (sizeof(T) == 4) {
        o.psq = (double)fma_of<T>(Pt, Pt, mul_of<T>(Pn, Pn));
        o.pabs = abs_of_sq<T>(o.psq);
    } else {
        o.psq = 0.0;
        o.pabs = SQ ? 0.0 : abs_of_pair(pn, pt);
    }
    o.rel_ok = 0; o.bad = 0;
    if (!apply_only && crit == CD_CONV_LOCAL) {
        const double d0 = (double)dPn, d1 = (double)dPt;
        const double s0 = __dadd_rn(pn, (double)r.P.x), s1 = __dadd_rn(pt, (double)r.P.y);
        const double d2 = sq2(d0, d1), s2 = sq2(s0, s1);
        o.rel_ok = d2 < __dmul_rn(alpha, s2);
        o.bad = !o.rel_ok && !(d2 <= __dmul_rn(__dmul_rn(alpha, ravg_prev), ravg_prev));
    }
    return o;
}

// Velocity of wall body n + 6 * packing + k.
__device__ __forceinline__ const double* wall_velocity(const CdGeom& g, const CdWork& w, int wid)
{
    const int t = wid - g.n;
    return (g.npk > 1) ? w.pk[t / 6].wall_vel + 3 * (t % 6) : g.wall_vel + 3 * t;
}

template <typename T>
__device__ __forceinline__ void wall_vel2(const CdGeom& g, const CdWork& w, int wid, typename Vec<T>::V4& vb)
{
    const double* u = wall_velocity(g, w, wid);
    vb.x = (T)u[0]; vb.y = (T)u[1]; vb.z = (T)0; vb.w = (T)0;
}

// VIEWS: the bodies' velocity records are the domain views r.vab, else their own.
// DEFER (FP64): the result's pabs is |P| of the thread's previous update,
// taken from its (P_n, P_t) `pend` after this update's velocity loads are
// issued; pn, pt hold this update's impulse.
// A 2D update computed but not yet stored: the two velocity records and the
// impulse, where they go.
template <typename T>
struct Staged2 {
    typename Vec<T>::V4 va, vb;
    typename Vec<T>::V2 P;
    int ia, ib, pos;
    bool wall, store_p;
};

template <typename T, bool VIEWS = false, bool DEFER = false>
__device__ __forceinline__ UpdOut stage2d(const CdGeom& g, const CdWork& w, int pos, const Rec<2, T>& r,
                                          bool apply_only, int crit, double alpha, double ravg_prev, double2 pend,
                                          Staged2<T>& st)
{
    typedef typename Vec<T>::V4 T4;
    const T4* V = (const T4*)w.V;
    st.ia = VIEWS ? r.vab.x : r.ab.x;
    st.ib = VIEWS ? r.vab.y : r.ab.y;
    st.pos = pos;
    st.store_p = !apply_only;
    st.wall = !cd_is_body(g, r.ab.y);   // kinematic wall
    st.va = V[st.ia];
    if (!st.wall) st.vb = V[st.ib];
    else wall_vel2<T>(g, w, r.ab.y, st.vb);
    Rec<2, T> rs = r;
    if constexpr (sizeof(T) == 8) load_static<2, T>(g, w, rs);
    const double prev = DEFER ? abs_of_pair(pend.x, pend.y) : 0.0;
    UpdOut o = core2d<T, DEFER>(g, rs, st.va, st.vb, st.wall, apply_only, crit, alpha, ravg_prev, st.P);
    if constexpr (DEFER) o.pabs = prev;
    if (!st.wall && r.ab.y >= g.n) {
        // a force-controlled wall moves along its normal only
        if (((r.ab.y - g.n) >> 1) == 0) st.vb.y = (T)0; else st.vb.x = (T)0;
        st.vb.z = (T)0;
    }
    return o;
}

template <typename T>
__device__ __forceinline__ void commit2d(const CdWork& w, const Staged2<T>& st)
{
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    T4* V = (T4*)w.V;
    V[st.ia] = st.va;
    if (!st.wall) V[st.ib] = st.vb;
    if (st.store_p) ((T2*)w.c_P)[st.pos] = st.P;
}

template <typename T, bool VIEWS = false, bool DEFER = false>
__device__ __forceinline__ UpdOut apply2d(const CdGeom& g, const CdWork& w, int pos, const Rec<2, T>& r,
                                          bool apply_only, int crit, double alpha, double ravg_prev,
                                          double2 pend = make_double2(0.0, 0.0))
{
    Staged2<T> st;
    const UpdOut o = stage2d<T, VIEWS, DEFER>(g, w, pos, r, apply_only, crit, alpha, ravg_prev, pend, st);
    commit2d<T>(w, st);
    return o;
}

// 3D: the same with the tangential impulse a vector, scaled onto the cone.
template <typename T, bool SQ = false>
__device__ __forceinline__ UpdOut core3d(const CdGeom& g, const Rec<3, T>& r, typename Vec<T>::V4& va,
                                         typename Vec<T>::V4& wa, typename Vec<T>::V4& vb, typename Vec<T>::V4& wb,
                                         bool wall, bool apply_only, int crit, double alpha, double ravg_prev,
                                         typename Vec<T>::V4& Pnew)
{
    // every operation written out, as in core2d
    const T nx = r.geo.x, ny = r.geo.y, nz = r.geo.z;
    T Pn, Ptx, Pty, Ptz, dPn, dtx, dty, dtz;
    if (apply_only) {
        Pn = r.P.x; Ptx = r.P.y; Pty = r.P.z; Ptz = r.P.w;
        dPn = Pn; dtx = Ptx; dty = Pty; dtz = Ptz;
    } else {
        const T mn = r.m.x, mt = r.m.y, b = r.geo.w;
        // relative velocity of the contact points: (vb - va) - (ra wa + rb wb) x n
        const T lx = fma_of<T>(r.sb.y, wb.x, mul_of<T>(r.sa.y, wa.x));
        const T ly = fma_of<T>(r.sb.y, wb.y, mul_of<T>(r.sa.y, wa.y));
        const T lz = fma_of<T>(r.sb.y, wb.z, mul_of<T>(r.sa.y, wa.z));
        const T gx = sub_of<T>(sub_of<T>(vb.x, va.x), fma_of<T>(ly, nz, -mul_of<T>(lz, ny)));
        const T gy = sub_of<T>(sub_of<T>(vb.y, va.y), fma_of<T>(lz, nx, -mul_of<T>(lx, nz)));
        const T gz = sub_of<T>(sub_of<T>(vb.z, va.z), fma_of<T>(lx, ny, -mul_of<T>(ly, nx)));
        const T un = fma_of<T>(gz, nz, fma_of<T>(gy, ny, mul_of<T>(gx, nx)));
        const T tx = fma_of<T>(-un, nx, gx), ty = fma_of<T>(-un, ny, gy), tz = fma_of<T>(-un, nz, gz);
        Pn = pos_part(fma_of<T>(-mn, add_of<T>(b, un), r.P.x));
        Ptx = fma_of<T>(-mt, tx, r.P.y);
        Pty = fma_of<T>(-mt, ty, r.P.z);
        Ptz = fma_of<T>(-mt, tz, r.P.w);
        const T lim = mul_of<T>(r.mu, Pn);
        const T q2 = fma_of<T>(Ptz, Ptz, fma_of<T>(Pty, Pty, mul_of<T>(Ptx, Ptx)));
        if (q2 > mul_of<T>(lim, lim)) {
            const T sc = mul_of<T>(lim, rsqrt(q2));   // onto the cone (q2 > lim^2 >= 0)
            Ptx = mul_of<T>(Ptx, sc); Pty = mul_of<T>(Pty, sc); Ptz = mul_of<T>(Ptz, sc);
        }
        dPn = sub_of<T>(Pn, r.P.x);
        dtx = sub_of<T>(Ptx, r.P.y); dty = sub_of<T>(Pty, r.P.z); dtz = sub_of<T>(Ptz, r.P.w);
    }
    const T dx = fma_of<T>(dPn, nx, dtx), dy = fma_of<T>(dPn, ny, dty), dz = fma_of<T>(dPn, nz, dtz);
    // n x dP
    const T cx = fma_of<T>(ny, dz, -mul_of<T>(nz, dy));
    const T cy = fma_of<T>(nz, dx, -mul_of<T>(nx, dz));
    const T cz = fma_of<T>(nx, dy, -mul_of<T>(ny, dx));
    va.x = fma_of<T>(-r.sa.x, dx, va.x); va.y = fma_of<T>(-r.sa.x, dy, va.y); va.z = fma_of<T>(-r.sa.x, dz, va.z);
    wa.x = fma_of<T>(-r.sa.z, cx, wa.x); wa.y = fma_of<T>(-r.sa.z, cy, wa.y); wa.z = fma_of<T>(-r.sa.z, cz, wa.z);
    if (!wall) {
        vb.x = fma_of<T>(r.sb.x, dx, vb.x); vb.y = fma_of<T>(r.sb.x, dy, vb.y); vb.z = fma_of<T>(r.sb.x, dz, vb.z);
        wb.x = fma_of<T>(-r.sb.z, cx, wb.x); wb.y = fma_of<T>(-r.sb.z, cy, wb.y); wb.z = fma_of<T>(-r.sb.z, cz, wb.z);
    }
    Pnew.x = Pn; Pnew.y = Ptx; Pnew.z = Pty; Pnew.w = Ptz;
    UpdOut o;
    const double pn = (double)Pn, px = (double)Ptx, py = (double)Pty, pz = (double)Ptz;
    o.pn = pn;
    o.pt = 0.0;
    if constexpr (sizeof(T) == 4)
        o.psq = (double)fma_of<T>(Ptz, Ptz, fma_of<T>(Pty, Pty, fma_of<T>(Ptx, Ptx, mul_of<T>(Pn, Pn))));
    else
        o.psq = __fma_rn(pz, pz, __fma_rn(py, py, __fma_rn(px, px, __dmul_rn(pn, pn))));
    o.pabs = SQ ? 0.0 : abs_of_sq<T>(o.psq);
    o.rel_ok = 0; o.bad = 0;
    if (!apply_only && crit == CD_CONV_LOCAL) {
        const double d0 = (double)dPn, d1 = (double)dtx, d2_ = (double)dty, d3 = (double)dtz;
        const double s0 = __dadd_rn(pn, (double)r.P.x), s1 = __dadd_rn(px, (double)r.P.y);
        const double s2_ = __dadd_rn(py, (double)r.P.z), s3 = __dadd_rn(pz, (double)r.P.w);
        const double d2 = __fma_rn(d3, d3, __fma_rn(d2_, d2_, __fma_rn(d1, d1, __dmul_rn(d0, d0))));
        const double s2 = __fma_rn(s3, s3, __fma_rn(s2_, s2_, __fma_rn(s1, s1, __dmul_rn(s0, s0))));
        o.rel_ok = d2 < __dmul_rn(alpha, s2);
        o.bad = !o.rel_ok && !(d2 <= __dmul_rn(__dmul_rn(alpha, ravg_prev), ravg_prev));
    }
    return o;
}

template <typename T>
__device__ __forceinline__ void wall_vel3(const CdGeom& g, const CdWork& w, int wid, typename Vec<T>::V4& vb,
                                          typename Vec<T>::V4& wb)
{
    const double* u = wall_velocity(g, w, wid);
    vb.x = (T)u[0]; vb.y = (T)u[1]; vb.z = (T)u[2]; vb.w = (T)0;
    wb.x = wb.y = wb.z = wb.w = (T)0;
}

template <typename T, bool VIEWS = false, bool DEFER = false>
__device__ __forceinline__ UpdOut apply3d(const CdGeom& g, const CdWork& w, int pos, const Rec<3, T>& r,
                                          bool apply_only, int crit, double alpha, double ravg_prev,
                                          double2 pend = make_double2(0.0, 0.0))
{
    typedef typename Vec<T>::V4 T4;
    T4* V = (T4*)w.V;
    const int ia = VIEWS ? r.vab.x : r.ab.x, ib = VIEWS ? r.vab.y : r.ab.y;
    const bool wall = !cd_is_body(g, r.ab.y);   // kinematic wall
    T4 va = V[2 * ia], wa = V[2 * ia + 1];
    T4 vb, wb;
    if (!wall) { vb = V[2 * ib]; wb = V[2 * ib + 1]; }
    else wall_vel3<T>(g, w, r.ab.y, vb, wb);
    Rec<3, T> rs = r;
    if constexpr (sizeof(T) == 8) load_static<3, T>(g, w, rs);
    const double prev = DEFER ? abs_of_pair(pend.x, pend.y) : 0.0;
    T4 Pnew;
    UpdOut o = core3d<T, DEFER>(g, rs, va, wa, vb, wb, wall, apply_only, crit, alpha, ravg_prev, Pnew);
    if constexpr (DEFER) o.pabs = prev;
    V[2 * ia] = va; V[2 * ia + 1] = wa;
    if (!wall) {
        if (r.ab.y >= g.n) {
            // a force-controlled wall moves along its normal only
            const int ax = (r.ab.y - g.n) >> 1;
            if (ax != 0) vb.x = (T)0;
            if (ax != 1) vb.y = (T)0;
            if (ax != 2) vb.z = (T)0;
            wb.x = wb.y = wb.z = (T)0;
        }
        V[2 * ib] = vb; V[2 * ib + 1] = wb;
    }
    if (!apply_only) ((T4*)w.c_P)[pos] = Pnew;
    return o;
}

template <int DIM, typename T, bool VIEWS = false, bool DEFER = false>
__device__ __forceinline__ UpdOut apply_rec(const CdGeom& g, const CdWork& w, int pos, const Rec<DIM, T>& r,
                                            bool apply_only, int crit, double alpha, double ravg_prev,
                                            double2 pend = make_double2(0.0, 0.0))
{
    if constexpr (DIM == 2)
        return apply2d<T, VIEWS, DEFER>(g, w, pos, r, apply_only, crit, alpha, ravg_prev, pend);
    else return apply3d<T, VIEWS, DEFER>(g, w, pos, r, apply_only, crit, alpha, ravg_prev, pend);
}

// Loads this thread's first record of colour k (if it has one) into nxt.
template <int DIM, typename T, bool VIEWS = false>
__device__ __forceinline__ void prefetch_first(const CdGeom& g, const CdWork& w, const int* s_off, int k,
                                               Rec<DIM, T>& nxt)
{
    const CdSpan sq = cd_colour_span(s_off[k], s_off[k + 1]);
    if (sq.p < sq.end) load_rec<DIM, T, VIEWS>(g, w, sq.p, nxt);
}

// Loads this thread's first record of phase k: of the colour class, or of
// this block's first list of the merged phase.
template <int DIM, typename T, int MODE>
__device__ __forceinline__ void prefetch_any(const CdGeom& g, const CdWork& w, const int* s_off, int k,
                                             Rec<DIM, T>& nxt, const MgInfo& mg)
{
    if constexpr (MODE == CD_SWEEP_MERGE) {
        if (mg.on && k == mg.klast) {
            // item q = threadIdx.x of the block's lists taken in turn
            int q = (int)threadIdx.x;
            for (int m = 0; m < mg.M; ++m) {
                const int cnt = mg.lst[2 * m + 1] - mg.lst[2 * m];
                if (q < cnt) {
                    load_rec<DIM, T>(g, w, w.mg_list[mg.lst[2 * m] + q], nxt);
                    break;
                }
                q -= cnt;
            }
            return;
        }
    }
    prefetch_first<DIM, T, MODE == CD_SWEEP_DOMAINS>(g, w, s_off, k, nxt);
}

// One colour phase for this thread: its first contact's record was loaded
// into `nxt` before the barrier (if it has one); the rest are loaded inline.
// Afterwards `nxt` holds the first record of colour `knext` (prefetch).
// `pend` carries (P_n, P_t) of the thread's last update whose magnitude is
// not yet in acc[0] (zeros if none) from phase to phase; the caller adds it
// before the block sum at the end of a pass.
template <int DIM, typename T, int MODE>
__device__ __forceinline__ void colour_phase(const CdGeom& g, const CdWork& w, const int* s_off, int k, int knext,
                                             int tid, int stride, Rec<DIM, T>& nxt, bool apply_only, int crit,
                                             double alpha, double ravg_prev, double (&acc)[3], double2& pend,
                                             const MgInfo& mg, bool skip_first = false)
{
    constexpr bool MIXED = (MODE == CD_SWEEP_MIXED);
    constexpr bool VIEWS = (MODE == CD_SWEEP_DOMAINS);
    // FP64 2D only: FP32 takes its square root on the fast pipe, and in 3D the
    // extra live value spills
    constexpr bool DEFER = (DIM == 2) && std::is_same<T, double>::value;
    if constexpr (MODE == CD_SWEEP_MERGE) {
        if (mg.on && k == mg.klast) {
            // the chains' contacts of colour K-M, a block barrier, those of K-M+1, ...
            const int t = (int)threadIdx.x, bd = (int)blockDim.x;
            int base = 0;   // items of the earlier lists
            for (int m = 0; m < mg.M; ++m) {
                const int l0 = mg.lst[2 * m], cnt = mg.lst[2 * m + 1] - l0;
                int q0 = t;
                if (q0 < base) q0 += ((base - q0 + bd - 1) / bd) * bd;   // this thread's first item of list m
                for (int q = q0; q < base + cnt; q += bd) {
                    const int p = w.mg_list[l0 + (q - base)];
                    UpdOut o;
                    if (q == t) {
                        o = apply_rec<DIM, T, false, DEFER>(g, w, p, nxt, apply_only, crit, alpha, ravg_prev, pend);
                    } else {
                        Rec<DIM, T> r;
                        load_rec<DIM, T>(g, w, p, r);
                        o = apply_rec<DIM, T, false, DEFER>(g, w, p, r, apply_only, crit, alpha, ravg_prev, pend);
                    }
                    acc[0] += o.pabs;
                    if (DEFER) pend = make_double2(o.pn, o.pt);
                    if (crit == CD_CONV_LOCAL) { acc[1] += (double)o.rel_ok; acc[2] += (double)o.bad; }
                }
                base += cnt;
                if (m + 1 < mg.M) __syncthreads();
            }
            if (knext >= 0) prefetch_any<DIM, T, MODE>(g, w, s_off, knext, nxt, mg);
            return;
        }
    }
    const CdSpan sp = cd_colour_span(s_off[k], s_off[k + 1]);
    const int end = sp.end;
    int p = sp.p;
    const bool mixed = MIXED && !apply_only;   // parallel contacts were done in their own phase
    if (p < end) {
        // skip_first: this thread's first update of the phase was staged and
        // stored before the phase (the first colour of a sweep, see k_sweep)
        if (!skip_first && !(mixed && cd_is_parallel(g.par_p, g.seed, cd_key(nxt.ab.x, nxt.ab.y), mg.draw))) {
            UpdOut o = apply_rec<DIM, T, VIEWS, DEFER>(g, w, p, nxt, apply_only, crit, alpha, ravg_prev, pend);
            acc[0] += o.pabs;
            if (DEFER) pend = make_double2(o.pn, o.pt);
            if (crit == CD_CONV_LOCAL) { acc[1] += (double)o.rel_ok; acc[2] += (double)o.bad; }
        }
        for (p += blockDim.x; p < end; p += blockDim.x) {
            Rec<DIM, T> r;
            load_rec<DIM, T, VIEWS>(g, w, p, r);
            if (mixed && cd_is_parallel(g.par_p, g.seed, cd_key(r.ab.x, r.ab.y), mg.draw)) continue;
            UpdOut o = apply_rec<DIM, T, VIEWS, DEFER>(g, w, p, r, apply_only, crit, alpha, ravg_prev, pend);
            acc[0] += o.pabs;
            if (DEFER) pend = make_double2(o.pn, o.pt);
            if (crit == CD_CONV_LOCAL) { acc[1] += (double)o.rel_ok; acc[2] += (double)o.bad; }
        }
    }
    if (knext >= 0) prefetch_any<DIM, T, MODE>(g, w, s_off, knext, nxt, mg);
    (void)tid; (void)stride;
}

// Epilogue shared by both sweep kernels: impulses back to key order (FP64),
// wall forces and the solve statistics.
template <int DIM, typename T>
__device__ __forceinline__ void finish_solve(const CdGeom& g, const CdWork& w, int nc, int nb, int tid, int stride,
                                             unsigned long long& epoch, int sweeps, int converged, double resid,
                                             double ravg, double (*s_red)[3], double& s_bc)
{
    CdCtrl* ctrl = w.ctrl;
    double wsum[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    for (int p = tid; p < nc; p += stride) {
        int c = w.perm[p];
        int2 ab = w.c_ab[p];
        double pn;
        if (DIM == 2) {
            T2 P = ((const T2*)w.c_P)[p];
            pn = (double)P.x;
            w.Pk[2 * c] = (double)P.x;
            w.Pk[2 * c + 1] = (double)P.y;
        } else {
            T4 P = ((const T4*)w.c_P)[p];
            pn = (double)P.x;
            w.Pk[4 * c] = (double)P.x;
            w.Pk[4 * c + 1] = (double)P.y;
            w.Pk[4 * c + 2] = (double)P.z;
            w.Pk[4 * c + 3] = (double)P.w;
        }
        if (ab.y >= g.n) {
            int k = ab.y - g.n;
#pragma unroll
            for (int q = 0; q < 6; ++q) if (q == k) wsum[q] += pn;
        }
    }
    {
        double a[3] = {wsum[0], wsum[1], wsum[2]};
        block_sum<3>(a, s_red);
        double b3[3] = {wsum[3], wsum[4], wsum[5]};
        block_sum<3>(b3, s_red);
        if (threadIdx.x == 0) {
            for (int q = 0; q < 3; ++q) w.wpart[q * nb + blockIdx.x] = a[q];
            for (int q = 0; q < 3; ++q) w.wpart[(3 + q) * nb + blockIdx.x] = b3[q];
        }
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    if (blockIdx.x == 0) {
        double wf[6];
        for (int q = 0; q < 6; ++q) wf[q] = grid_total(w.wpart + q * nb, nb, &s_bc);
        if (threadIdx.x == 0) {
            for (int q = 0; q < 6; ++q) ctrl->wall_force[q] = wf[q] / g.dt;
            ctrl->sweeps = sweeps;
            ctrl->mg_prev = sweeps + 1;
            ctrl->converged = converged;
            ctrl->residual = resid;
            ctrl->r_avg = ravg;
            ctrl->steps_done += 1;
            ctrl->total_sweeps += sweeps;
            ctrl->total_updates += (long long)sweeps * (long long)nc;
            if (sweeps > ctrl->max_sweeps_step) ctrl->max_sweeps_step = sweeps;
            if (!converged) ctrl->n_not_conv += 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Mixed update (Sec. 2.3).  Parallel contacts compute their new impulse from
// the velocities at the start of the sweep (no velocity change yet) and keep
// the change; after the sequential colours each particle adds the changes of
// its parallel contacts in ascending key order.
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__device__ __forceinline__ UpdOut par_compute(const CdGeom& g, const CdWork& w, int p, const Rec<DIM, T>& r, int crit,
                                              double alpha, double ravg_prev)
{
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    const T4* V = (const T4*)w.V;
    const bool wall = r.ab.y >= g.n;
    const int c = w.perm[p];
    UpdOut o;
    Rec<DIM, T> rs = r;
    if constexpr (sizeof(T) == 8) load_static<DIM, T>(g, w, rs);
    if constexpr (DIM == 2) {
        T4 va = V[r.ab.x], vb;
        if (!wall) vb = V[r.ab.y];
        else wall_vel2<T>(g, w, r.ab.y, vb);
        T2 Pnew;
        o = core2d<T>(g, rs, va, vb, wall, false, crit, alpha, ravg_prev, Pnew);
        ((T2*)w.c_P)[p] = Pnew;
        w.c_dpar[2 * c] = (double)(Pnew.x - r.P.x);
        w.c_dpar[2 * c + 1] = (double)(Pnew.y - r.P.y);
    } else {
        T4 va = V[2 * r.ab.x], wa = V[2 * r.ab.x + 1], vb, wb;
        if (!wall) { vb = V[2 * r.ab.y]; wb = V[2 * r.ab.y + 1]; }
        else wall_vel3<T>(g, w, r.ab.y, vb, wb);
        T4 Pnew;
        o = core3d<T>(g, rs, va, wa, vb, wb, wall, false, crit, alpha, ravg_prev, Pnew);
        ((T4*)w.c_P)[p] = Pnew;
        w.c_dpar[4 * c] = (double)(Pnew.x - r.P.x);
        w.c_dpar[4 * c + 1] = (double)(Pnew.y - r.P.y);
        w.c_dpar[4 * c + 2] = (double)(Pnew.z - r.P.z);
        w.c_dpar[4 * c + 3] = (double)(Pnew.w - r.P.w);
    }
    return o;
}

template <int DIM, typename T>
__device__ __forceinline__ void par_apply(const CdGeom& g, const CdWork& w, int tid, int stride, long long draw)
{
    typedef typename Vec<T>::V4 T4;
    T4* V = (T4*)w.V;
    const T4* S = (const T4*)w.S;
    for (int i = tid; i < g.n; i += stride) {
        const int e = w.p2c_off[i + 1];
        bool any = false;
        T4 v, om;
        const T4 si = S[i];
        for (int q = w.p2c_off[i]; q < e; ++q) {
            const int c = w.p2c[q];
            const int2 ab = w.pairs[c];
            if (!cd_is_parallel(g.par_p, g.seed, cd_key(ab.x, ab.y), draw)) continue;
            if (!any) {
                any = true;
                if (DIM == 2) v = V[i];
                else { v = V[2 * i]; om = V[2 * i + 1]; }
            }
            const T sign = (ab.x == i) ? (T)-1 : (T)1;
            const T nx = (T)w.nrm[3 * c], ny = (T)w.nrm[3 * c + 1], nz = (T)w.nrm[3 * c + 2];
            if (DIM == 2) {
                const T dPn = (T)w.c_dpar[2 * c], dPt = (T)w.c_dpar[2 * c + 1];
                const T dx = dPn * nx - dPt * ny, dy = dPn * ny + dPt * nx;
                v.x += sign * si.x * dx; v.y += sign * si.x * dy;
                v.z -= si.z * dPt;
            } else {
                const T dPn = (T)w.c_dpar[4 * c];
                const T dx = dPn * nx + (T)w.c_dpar[4 * c + 1];
                const T dy = dPn * ny + (T)w.c_dpar[4 * c + 2];
                const T dz = dPn * nz + (T)w.c_dpar[4 * c + 3];
                const T cx = ny * dz - nz * dy, cy = nz * dx - nx * dz, cz = nx * dy - ny * dx;
                v.x += sign * si.x * dx; v.y += sign * si.x * dy; v.z += sign * si.x * dz;
                om.x -= si.z * cx; om.y -= si.z * cy; om.z -= si.z * cz;
            }
        }
        if (any) {
            if (DIM == 2) store_xyz_plain<T>(V + i, v);
            else { store_xyz_plain<T>(V + 2 * i, v); V[2 * i + 1] = om; }
        }
    }
}

// ---------------------------------------------------------------------------
// Domain-wise update (Sec. 3.1).  Each contact updates the velocity records
// of its domain (c_vab).  Before the first pass every view record takes its
// particle's velocity; after every pass (the starting impulses, then each
// sweep) a particle with views gets v0 + (v_home - v0) + sum over its views
// in ascending domain order of (v_view - v0), v0 being the velocity of the
// pass start, and every view starts the next pass from that sum.
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__device__ __forceinline__ void dom_init(const CdGeom& g, const CdWork& w, int tid, int stride)
{
    typedef typename Vec<T>::V4 T4;
    constexpr int RW = (DIM == 2) ? 1 : 2;   // records per body
    T4* V = (T4*)w.V;
    T4* V0 = (T4*)w.V0;
    const int nv = w.view_off[g.n], base = cd_view_base(g);
    for (int q = tid; q < nv; q += stride) {
        const int i = w.view_owner[q];
#pragma unroll
        for (int h = 0; h < RW; ++h) {
            const T4 x = V[RW * i + h];
            V[RW * (base + q) + h] = x;
            V0[RW * q + h] = x;
        }
    }
}

template <int DIM, typename T>
__device__ __forceinline__ void dom_combine(const CdGeom& g, const CdWork& w, int tid, int stride)
{
    typedef typename Vec<T>::V4 T4;
    constexpr int RW = (DIM == 2) ? 1 : 2;
    T4* V = (T4*)w.V;
    T4* V0 = (T4*)w.V0;
    const int nv = w.view_off[g.n], base = cd_view_base(g);
    for (int q = tid; q < nv; q += stride) {
        const int i = w.view_owner[q];
        if (q != w.view_off[i]) continue;   // one thread per particle: its first view
        const int e = w.view_off[i + 1];
#pragma unroll
        for (int h = 0; h < RW; ++h) {
            const T4 s0 = V0[RW * q + h];
            T4 x = V[RW * i + h];
            T sx = s0.x + (x.x - s0.x), sy = s0.y + (x.y - s0.y), sz = s0.z + (x.z - s0.z);
            for (int u = q; u < e; ++u) {
                const T4 a = V[RW * (base + u) + h];
                sx = sx + (a.x - s0.x);
                sy = sy + (a.y - s0.y);
                sz = sz + (a.z - s0.z);
            }
            x.x = sx; x.y = sy; x.z = sz;
            V[RW * i + h] = x;
            for (int u = q; u < e; ++u) {
                V[RW * (base + u) + h] = x;
                V0[RW * u + h] = x;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The persistent sweep kernel
// ---------------------------------------------------------------------------
// MODE: CD_SWEEP_PLAIN, CD_SWEEP_MIXED (the mixed update of Sec. 2.3,
// params.parallel_p > 0) or CD_SWEEP_DOMAINS (the domain-wise update of
// Sec. 3.1, params.domains); each variant carries only its own code.
template <int DIM, typename T, int MODE>
__global__ void __launch_bounds__(CD_SWEEP_THREADS, 1)
k_sweep(CdGeom g, CdWork w, int crit, double alpha, int max_sweeps)
{
    constexpr bool MIXED = (MODE == CD_SWEEP_MIXED);
    constexpr bool VIEWS = (MODE == CD_SWEEP_DOMAINS);
    __shared__ int s_off[CD_KMAX + 1];
    __shared__ double s_red[CD_SWEEP_THREADS / 32][3];
    __shared__ double s_bc;
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    const int nc = ctrl->nc;
    int K = ctrl->ncolours;
    const int nb = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    unsigned long long epoch = 0;
    for (int k = threadIdx.x; k <= CD_KMAX; k += blockDim.x) s_off[k] = w.colour_off[k];
    MgInfo mg;
    mg.on = 0; mg.klast = -1; mg.M = 0; mg.lst = nullptr; mg.draw = -1;
    __shared__ int s_mgl[2 * CD_MG_MAXC];
    if constexpr (MODE == CD_SWEEP_MERGE) {
        const int M = ctrl->merge;
        if (M >= 2 && M <= CD_MG_MAXC && nb == g.merge_blocks) {
            // the M last colours run as one phase (lists built for this grid)
            mg.on = 1;
            mg.M = M;
            K -= M - 1;
            mg.klast = K - 1;
            const int b = blockIdx.x;
            if (threadIdx.x < 2 * M) {
                const int m = threadIdx.x >> 1;
                s_mgl[threadIdx.x] = w.mg_boff[m * nb + b + (threadIdx.x & 1)];
            }
            mg.lst = s_mgl;
        }
    }
    __syncthreads();

    int sweeps = 0, converged = (nc == 0);
    double resid = 0.0, ravg = 0.0, ravg_prev = 0.0;
    if (nc > 0) {
        if constexpr (VIEWS) {
            dom_init<DIM, T>(g, w, tid, stride);
            if (!cd_grid_sync(ctrl, nb, epoch)) return;
        }
        Rec<DIM, T> nxt;
        prefetch_any<DIM, T, MODE>(g, w, s_off, 0, nxt, mg);
        // starting impulses, colour by colour
        double acc[3] = {0.0, 0.0, 0.0};
        double2 pend = make_double2(0.0, 0.0);   // this thread's last impulse not yet in the residual sum
        for (int k = 0; k < K; ++k) {
            colour_phase<DIM, T, MODE>(g, w, s_off, k, (k + 1 < K) ? k + 1 : 0, tid, stride, nxt, true, crit, alpha,
                                       0.0, acc, pend, mg);
            if (k == K - 1) {
                acc[0] += abs_of_pair(pend.x, pend.y);
                pend = make_double2(0.0, 0.0);
                block_sum<3>(acc, s_red, 1);
                if (threadIdx.x == 0) w.partials[blockIdx.x] = acc[0];
            }
            if (!cd_grid_sync(ctrl, nb, epoch)) return;
        }
        if constexpr (VIEWS) {
            dom_combine<DIM, T>(g, w, tid, stride);
            if (!cd_grid_sync(ctrl, nb, epoch)) return;
        }
        ravg_prev = grid_total(w.partials, nb, &s_bc) / (double)nc;
        ravg = ravg_prev;

        // 2D plain and merged schedules under the global tests: while the last
        // warp of each block runs the convergence test of sweep j, the other
        // threads compute their first update of sweep j + 1 (colour 0, its
        // record prefetched) into registers and store it only if the test
        // says continue.  The same updates in the same order: bits unchanged.
        constexpr bool SPEC_OK = (DIM == 2) && !MIXED && !VIEWS;
        const bool spec_on = SPEC_OK && crit != CD_CONV_LOCAL && !(mg.on && mg.klast == 0);
        bool spec_done = false;   // this thread's first colour-0 update of the coming sweep is stored
        double carry = 0.0;       // its residual term (the first term of the sweep's sum)
        while (!converged && sweeps < max_sweeps) {
            const int buf = (sweeps & 1) ? 0 : 1;   // alternate with the buffer of the previous sweep
            double* part = w.partials + (size_t)buf * 3 * nb;
            double a3[3] = {carry, 0.0, 0.0};
            carry = 0.0;
            const bool mixed = MIXED;
            if (MIXED && g.par_redraw) mg.draw = sweeps;   // this iteration step's parallel subset
            if (mixed) {
                for (int p = tid; p < nc; p += stride) {
                    Rec<DIM, T> r;
                    load_rec<DIM, T>(g, w, p, r);
                    if (!cd_is_parallel(g.par_p, g.seed, cd_key(r.ab.x, r.ab.y), mg.draw)) continue;
                    UpdOut o = par_compute<DIM, T>(g, w, p, r, crit, alpha, ravg_prev);
                    a3[0] += o.pabs;
                    if (crit == CD_CONV_LOCAL) { a3[1] += (double)o.rel_ok; a3[2] += (double)o.bad; }
                }
                if (!cd_grid_sync(ctrl, nb, epoch)) return;
                // the prefetched record of colour 0 may belong to a parallel contact whose
                // impulse just changed: reload it
                const CdSpan s0 = cd_colour_span(s_off[0], s_off[1]);
                if (s0.p < s0.end) load_rec<DIM, T>(g, w, s0.p, nxt);
            }
            for (int k = 0; k < K; ++k) {
                // no prefetch inside the phase: it is issued after the barrier arrival
                // below, so that the arriving thread's fence does not wait for it
                colour_phase<DIM, T, MODE>(g, w, s_off, k, -1, tid, stride, nxt, false, crit, alpha, ravg_prev, a3,
                                           pend, mg, k == 0 && spec_done);
                if (k == K - 1) {
                    // (a thread without a pending impulse adds nothing: skip the FP64 work)
                    if ((__double_as_longlong(pend.x) | __double_as_longlong(pend.y)) != 0)
                        a3[0] += abs_of_pair(pend.x, pend.y);
                    pend = make_double2(0.0, 0.0);
                }
                if (mixed && k == K - 1) {
                    if (!cd_grid_sync(ctrl, nb, epoch)) return;
                    par_apply<DIM, T>(g, w, tid, stride, mg.draw);
                }
                if (k == K - 1) {
                    block_sum<3>(a3, s_red, test_values(crit));
                    if (threadIdx.x == 0) {
                        part[blockIdx.x] = a3[0];
                        part[nb + blockIdx.x] = a3[1];
                        part[2 * nb + blockIdx.x] = a3[2];
                    }
                }
                const unsigned old = cd_grid_arrive(ctrl, nb);
                if (!mixed || k + 1 < K) prefetch_any<DIM, T, MODE>(g, w, s_off, (k + 1 < K) ? k + 1 : 0, nxt, mg);
                if (!cd_grid_wait(ctrl, old, epoch)) return;
            }
            if constexpr (VIEWS) {
                dom_combine<DIM, T>(g, w, tid, stride);
                if (!cd_grid_sync(ctrl, nb, epoch)) return;
            }
            ++sweeps;
            spec_done = false;
            if constexpr (SPEC_OK) {
                constexpr bool DEFER = std::is_same<T, double>::value;
                Staged2<T> st;
                bool staged = false;
                if (spec_on && sweeps < max_sweeps) {
                    const CdSpan s0 = cd_colour_span(s_off[0], s_off[1]);
                    if (s0.p < s0.end) {
                        // pend is (0, 0) here (the last phase added it to the sum), so
                        // the staged update's own residual term is 0 under DEFER
                        (void)stage2d<T, false, DEFER>(g, w, s0.p, nxt, false, crit, alpha, ravg_prev, pend, st);
                        staged = true;
                    }
                }
                sweep_test(part, nb, nc, crit, alpha, ravg_prev, ravg, resid, converged, s_red[0]);
                if (staged && !converged) {
                    commit2d<T>(w, st);
                    spec_done = true;
                    if constexpr (DEFER) {
                        pend = make_double2((double)st.P.x, (double)st.P.y);   // its |P| joins the sum later
                    } else {
                        // |P| of the update, as core2d takes it in this precision
                        carry = abs_of_sq<T>((double)fma_of<T>(st.P.y, st.P.y, mul_of<T>(st.P.x, st.P.x)));
                    }
                }
            } else {
                sweep_test(part, nb, nc, crit, alpha, ravg_prev, ravg, resid, converged, s_red[0]);
            }
            ravg_prev = ravg;
        }
    }

    finish_solve<DIM, T>(g, w, nc, nb, tid, stride, epoch, sweeps, converged, resid, ravg, s_red, s_bc);
}

// ---------------------------------------------------------------------------
// Batched systems: independent packings share the colour phases (so each
// grid barrier is amortised over all of them) but each has its own
// convergence test.  After a sweep every block reduces |P| over the
// contiguous key-order contact range of the packings it owns (fixed order:
// deterministic), decides convergence, and a converged packing's contacts are
// skipped from the next sweep on, exactly as if it were solved alone.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pk_reduce(const CdGeom& g, const CdWork& w, int sweep, int crit, double alpha,
                                          int* act_slot, int* act_c_slot, double (*s_red)[3])
{
    for (int b = blockIdx.x; b < g.npk; b += gridDim.x) {
        double* st = w.pk_stats + CD_PKSTATS * b;
        if (sweep >= 0 && cd_ld_volatile_int(&w.pk_done[b])) continue;
        const int c0 = w.pk_coff[b], c1 = w.pk_coff[b + 1];
        double a3[3] = {0.0, 0.0, 0.0};
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            a3[0] += w.c_abs[c];
            if (crit == CD_CONV_LOCAL && sweep >= 0) {
                int f = w.c_flag[c];
                a3[1] += (double)(f & 1);
                a3[2] += (double)((f >> 1) & 1);
            }
        }
        block_sum<3>(a3, s_red, (crit == CD_CONV_LOCAL && sweep >= 0) ? 3 : 1);
        if (threadIdx.x == 0) {
            const int ncb = c1 - c0;
            const double R = (ncb > 0) ? a3[0] / (double)ncb : 0.0;
            if (sweep < 0) {
                st[PKS_SWEEPS] = 0.0;
                st[PKS_CONV] = (ncb == 0) ? 1.0 : 0.0;
                st[PKS_RESID] = 0.0;
                st[PKS_RAVG] = R;
                st[PKS_RPREV] = R;
                st[PKS_NC] = (double)ncb;
                w.pk_done[b] = (ncb == 0) ? 1 : 0;
            } else {
                const double Rp = st[PKS_RPREV], den = R + Rp;
                double resid;
                int conv;
                if (crit == CD_CONV_GLOBAL_REL) {
                    resid = (den > 0.0) ? fabs(R - Rp) / den : (den == 0.0 ? 0.0 : den);
                    conv = resid < alpha;
                } else if (crit == CD_CONV_GLOBAL_SQ) {
                    double q = (den > 0.0) ? (R - Rp) / den : (den == 0.0 ? 0.0 : den);
                    resid = q * q;
                    conv = resid < alpha;
                } else if (crit == CD_CONV_LOCAL) {
                    resid = (ncb > 0) ? (double)(ncb - (long long)a3[1]) / (double)ncb : 0.0;
                    conv = (10.0 * a3[1] >= 9.0 * (double)ncb) && a3[2] == 0.0;
                } else {
                    resid = (den > 0.0) ? fabs(R - Rp) / den : (den == 0.0 ? 0.0 : den);
                    conv = 0;
                }
                st[PKS_SWEEPS] = (double)(sweep + 1);
                st[PKS_RESID] = resid;
                st[PKS_RAVG] = R;
                st[PKS_RPREV] = R;
                if (conv) {
                    st[PKS_CONV] = 1.0;
                    w.pk_done[b] = 1;
                } else {
                    atomicAdd(act_slot, 1);
                    atomicAdd(act_c_slot, ncb);
                }
            }
        }
        __syncthreads();
    }
}

// Exclusive scan of a 0/1 flag over the block (ballot per warp, warp totals in
// shared memory); returns the flags before this thread, *total the block's sum.
__device__ __forceinline__ int block_excl_scan01(int f, int* s_warp, int* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    const int in_warp = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) s_warp[wid] = __popc(m);
    __syncthreads();
    int before = 0, tot = 0;
    for (int q = 0; q < nw; ++q) {
        const int c = s_warp[q];
        if (q < wid) before += c;
        tot += c;
    }
    __syncthreads();
    *total = tot;
    return before + in_warp;
}

// Drops the contacts of converged packings from the colour-order arrays: a
// stable partition into the second set of arrays, copied back to the front of
// the first, so that later sweeps spread only the active contacts over the
// grid.  A dropped contact's final impulse goes back to key order here.
// Colour order and the updates themselves are unchanged, so results are
// identical.  Returns the new number of positions (same in every block).
template <int DIM, typename T>
__device__ __forceinline__ int compact_batch(const CdGeom& g, const CdWork& w, int nact, int K, int* s_off,
                                             unsigned long long& epoch, bool& ok)
{
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    __shared__ int s_warp[CD_SWEEP_THREADS / 32];
    __shared__ int s_base;
    CdCtrl* ctrl = w.ctrl;
    const int nb = gridDim.x;
    const int chunk = (nact + nb - 1) / nb;
    const int lo = min((int)blockIdx.x * chunk, nact), hi = min(lo + chunk, nact);
    auto keep = [&](int p) { return cd_ld_volatile_int(&w.pk_done[w.pack_of[w.c_ab[p].x]]) == 0; };
    int cnt = 0;
    for (int p = lo + (int)threadIdx.x; p < hi; p += blockDim.x) cnt += keep(p) ? 1 : 0;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_warp[q];
        w.cmp_blk[blockIdx.x] = t;
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) { ok = false; return nact; }
    if (threadIdx.x == 0) {
        int b0 = 0, tot = 0;
        for (int q = 0; q < nb; ++q) {
            const int c = cd_ld_volatile_int(&w.cmp_blk[q]);
            if (q < (int)blockIdx.x) b0 += c;
            tot += c;
        }
        s_base = b0;
        if (blockIdx.x == 0)
            for (int k = 0; k <= K; ++k)
                if (s_off[k] == nact) w.cmp_off[k] = tot;
    }
    __syncthreads();
    int running = s_base;
    const int pw = (DIM == 2) ? 2 : 4;
    for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int p = t0 + (int)threadIdx.x;
        const int f = (p < hi) && keep(p);
        int tile_tot;
        const int ex = block_excl_scan01(f, s_warp, &tile_tot);
        if (p < hi) {
            for (int k = 0; k <= K; ++k)
                if (s_off[k] == p) w.cmp_off[k] = running + ex;
            if (f) {
                const int q = running + ex;
                w.c_ab2[q] = w.c_ab[p];
                ((T4*)w.c_geo2)[q] = ((const T4*)w.c_geo)[p];
                if constexpr (DIM == 2) {
                    ((T*)w.c_m2)[q] = ((const T*)w.c_m)[p];
                    ((T2*)w.c_P2)[q] = ((const T2*)w.c_P)[p];
                } else {
                    ((T2*)w.c_m2)[q] = ((const T2*)w.c_m)[p];
                    ((T4*)w.c_P2)[q] = ((const T4*)w.c_P)[p];
                }
                w.perm2[q] = w.perm[p];
            } else {
                const int c = w.perm[p];
                if constexpr (DIM == 2) {
                    const T2 P = ((const T2*)w.c_P)[p];
                    w.Pk[pw * c] = (double)P.x;
                    w.Pk[pw * c + 1] = (double)P.y;
                } else {
                    const T4 P = ((const T4*)w.c_P)[p];
                    w.Pk[pw * c] = (double)P.x; w.Pk[pw * c + 1] = (double)P.y;
                    w.Pk[pw * c + 2] = (double)P.z; w.Pk[pw * c + 3] = (double)P.w;
                }
            }
        }
        running += tile_tot;
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) { ok = false; return nact; }
    int tot = 0;
    for (int q = 0; q < nb; ++q) tot += cd_ld_volatile_int(&w.cmp_blk[q]);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += gridDim.x * blockDim.x) {
        w.c_ab[q] = w.c_ab2[q];
        ((T4*)w.c_geo)[q] = ((const T4*)w.c_geo2)[q];
        if constexpr (DIM == 2) {
            ((T*)w.c_m)[q] = ((const T*)w.c_m2)[q];
            ((T2*)w.c_P)[q] = ((const T2*)w.c_P2)[q];
        } else {
            ((T2*)w.c_m)[q] = ((const T2*)w.c_m2)[q];
            ((T4*)w.c_P)[q] = ((const T4*)w.c_P2)[q];
        }
        w.perm[q] = w.perm2[q];
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) { ok = false; return nact; }
    for (int k = threadIdx.x; k <= K; k += blockDim.x) s_off[k] = cd_ld_volatile_int(&w.cmp_off[k]);
    __syncthreads();
    return tot;
}

template <int DIM, typename T>
__global__ void __launch_bounds__(CD_SWEEP_THREADS, 1)
k_sweep_batch(CdGeom g, CdWork w, int crit, double alpha, int max_sweeps)
{
    __shared__ int s_off[CD_KMAX + 1];
    __shared__ double s_red[CD_SWEEP_THREADS / 32][3];
    CdCtrl* ctrl = w.ctrl;
    if (ctrl->skip) return;
    const int nc = ctrl->nc;
    const int K = ctrl->ncolours;
    const int nb = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    unsigned long long epoch = 0;
    for (int k = threadIdx.x; k <= CD_KMAX; k += blockDim.x) s_off[k] = w.colour_off[k];
    if (tid == 0)
        for (int q = 0; q < 6; ++q) w.act_cnt[q] = 0;
    __syncthreads();
    int nact = nc;   // positions still in the colour-order arrays

    // starting impulses, colour by colour
    for (int k = 0; k < K; ++k) {
        const CdSpan sp = cd_colour_span(s_off[k], s_off[k + 1]);
        for (int p = sp.p; p < sp.end; p += blockDim.x) {
            Rec<DIM, T> r;
            load_rec<DIM, T>(g, w, p, r);
            UpdOut o = apply_rec<DIM, T>(g, w, p, r, true, crit, alpha, 0.0);
            w.c_abs[w.perm[p]] = o.pabs;
        }
        if (!cd_grid_sync(ctrl, nb, epoch)) return;
    }
    pk_reduce(g, w, -1, crit, alpha, nullptr, nullptr, s_red);
    if (!cd_grid_sync(ctrl, nb, epoch)) return;

    for (int sweep = 0; sweep < max_sweeps && nc > 0; ++sweep) {
        if (tid == 0) { w.act_cnt[(sweep + 1) % 3] = 0; w.act_cnt[3 + (sweep + 1) % 3] = 0; }
        for (int k = 0; k < K; ++k) {
            const CdSpan sp = cd_colour_span(s_off[k], s_off[k + 1]);
            for (int p = sp.p; p < sp.end; p += blockDim.x) {
                Rec<DIM, T> r;
                load_rec<DIM, T>(g, w, p, r);
                if (w.pk_done[r.pk]) continue;
                const double rprev = (crit == CD_CONV_LOCAL) ? w.pk_stats[CD_PKSTATS * r.pk + PKS_RPREV] : 0.0;
                UpdOut o = apply_rec<DIM, T>(g, w, p, r, false, crit, alpha, rprev);
                const int c = w.perm[p];
                w.c_abs[c] = o.pabs;
                w.c_flag[c] = o.rel_ok | (o.bad << 1);
            }
            if (!cd_grid_sync(ctrl, nb, epoch)) return;
        }
        pk_reduce(g, w, sweep, crit, alpha, &w.act_cnt[sweep % 3], &w.act_cnt[3 + sweep % 3], s_red);
        if (!cd_grid_sync(ctrl, nb, epoch)) return;
        if (cd_ld_volatile_int(&w.act_cnt[sweep % 3]) == 0) break;
        // once a third of the positions belong to converged packings, drop them
        const int live = cd_ld_volatile_int(&w.act_cnt[3 + sweep % 3]);
        if (3 * (nact - live) >= nact && sweep + 1 < max_sweeps) {
            bool ok = true;
            nact = compact_batch<DIM, T>(g, w, nact, K, s_off, epoch, ok);
            if (!ok) return;
        }
    }

    // impulses back to key order (those of dropped contacts were written when dropped)
    typedef typename Vec<T>::V4 T4;
    typedef typename Vec<T>::V2 T2;
    for (int p = tid; p < nact; p += stride) {
        int c = w.perm[p];
        if (DIM == 2) {
            T2 P = ((const T2*)w.c_P)[p];
            w.Pk[2 * c] = (double)P.x;
            w.Pk[2 * c + 1] = (double)P.y;
        } else {
            T4 P = ((const T4*)w.c_P)[p];
            w.Pk[4 * c] = (double)P.x; w.Pk[4 * c + 1] = (double)P.y;
            w.Pk[4 * c + 2] = (double)P.z; w.Pk[4 * c + 3] = (double)P.w;
        }
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    // per-packing wall forces and the call's totals
    const int pw = (DIM == 2) ? 2 : 4;
    for (int b = blockIdx.x; b < g.npk; b += gridDim.x) {
        const int c0 = w.pk_coff[b], c1 = w.pk_coff[b + 1];
        double lo3[3] = {0.0, 0.0, 0.0}, hi3[3] = {0.0, 0.0, 0.0};
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            int bb = w.pairs[c].y;
            if (bb < g.n) continue;
            int k = (bb - g.n) % 6;
            double pn = w.Pk[pw * c];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (q == k) lo3[q] += pn;
                if (q + 3 == k) hi3[q] += pn;
            }
        }
        block_sum<3>(lo3, s_red);
        block_sum<3>(hi3, s_red);
        if (threadIdx.x == 0) {
            double* st = w.pk_stats + CD_PKSTATS * b;
            for (int q = 0; q < 3; ++q) {
                st[PKS_WF0 + q] = lo3[q] / g.dt;
                st[PKS_WF0 + 3 + q] = hi3[q] / g.dt;
            }
            const long long sw = (long long)st[PKS_SWEEPS];
            atomicAdd((unsigned long long*)&ctrl->total_updates, (unsigned long long)(sw * (long long)(c1 - c0)));
            atomicMax((unsigned long long*)&ctrl->max_sweeps_step, (unsigned long long)sw);
            if (st[PKS_CONV] == 0.0) atomicAdd((unsigned long long*)&ctrl->n_not_conv, 1ULL);
            if (b == 0) {
                for (int q = 0; q < 6; ++q) ctrl->wall_force[q] = st[PKS_WF0 + q];
                ctrl->r_avg = st[PKS_RAVG];
                ctrl->residual = st[PKS_RESID];
            }
        }
        __syncthreads();
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    if (tid == 0) {
        ctrl->steps_done += 1;
        long long tot = 0, mx = 0, open = 0;
        for (int b = 0; b < g.npk; ++b) {
            const long long sw = (long long)w.pk_stats[CD_PKSTATS * b + PKS_SWEEPS];
            tot += sw;
            if (sw > mx) mx = sw;
            if (w.pk_stats[CD_PKSTATS * b + PKS_CONV] == 0.0) ++open;
        }
        ctrl->total_sweeps += tot;
        ctrl->sweeps = mx;
        ctrl->converged = (open == 0);
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int grid_n(int n)
{
    int g = (n + CD_BLOCK - 1) / CD_BLOCK;
    return g < 1 ? 1 : (g > 4096 ? 4096 : g);
}

cudaError_t cd_launch_static(const CdGeom& g, const CdWork& w, const double* radius, const double* inv_m,
                             const double* inv_I, int precision, cudaStream_t s, int* nl)
{
    if (precision == CD_FP64)
        k_static<double><<<grid_n(g.n), CD_BLOCK, 0, s>>>(g, g.n, g.rotations, radius, inv_m, inv_I, (Vec<double>::V4*)w.S);
    else
        k_static<float><<<grid_n(g.n), CD_BLOCK, 0, s>>>(g, g.n, g.rotations, radius, inv_m, inv_I, (float4*)w.S);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t cd_launch_pack(const CdGeom& g, const CdWork& w, const double* vel, const double* omega,
                           const double* radius, const double* inv_m, const double* inv_I, const double* f_ext,
                           int free_flight, int precision, cudaStream_t s, int* nl)
{
    (void)radius; (void)inv_I;
    int gb = grid_n(g.n);
    if (g.dim == 2) {
        if (precision == CD_FP64) k_pack<2, double><<<gb, CD_BLOCK, 0, s>>>(g, w, vel, omega, inv_m, f_ext, free_flight);
        else k_pack<2, float><<<gb, CD_BLOCK, 0, s>>>(g, w, vel, omega, inv_m, f_ext, free_flight);
        ++*nl;
    } else {
        if (precision == CD_FP64) k_pack<3, double><<<gb, CD_BLOCK, 0, s>>>(g, w, vel, omega, inv_m, f_ext, free_flight);
        else k_pack<3, float><<<gb, CD_BLOCK, 0, s>>>(g, w, vel, omega, inv_m, f_ext, free_flight);
        ++*nl;
    }
    return cudaGetLastError();
}

cudaError_t cd_launch_unpack(const CdGeom& g, const CdWork& w, double* pos, double* vel, double* omega,
                             double* theta, int integrate, int precision, cudaStream_t s, int* nl)
{
    int gb = grid_n(g.n);
    if (g.dim == 2) {
        if (precision == CD_FP64) k_unpack<2, double><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, vel, omega, theta, integrate);
        else k_unpack<2, float><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, vel, omega, theta, integrate);
        ++*nl;
    } else {
        if (precision == CD_FP64) k_unpack<3, double><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, vel, omega, theta, integrate);
        else k_unpack<3, float><<<gb, CD_BLOCK, 0, s>>>(g, w, pos, vel, omega, theta, integrate);
        ++*nl;
    }
    return cudaGetLastError();
}

// Kernel of each schedule: 0 colour barrier, 3 batched, 4 mixed update,
// 5 domain-wise update, 6 merged last colours.
static int sweep_kind(const CdGeom& g)
{
    if (g.npk > 1) return 3;
    if (g.par_p > 0.0) return 4;
    if (g.ndom_total > 1) return 5;
    if (g.merge_last) return 6;
    return 0;
}

static const void* sweep_fn(int dim, int precision, int kind)
{
    if (kind == 6) {
        if (dim == 2)
            return precision == CD_FP64 ? (const void*)k_sweep<2, double, CD_SWEEP_MERGE>
                                        : (const void*)k_sweep<2, float, CD_SWEEP_MERGE>;
        return precision == CD_FP64 ? (const void*)k_sweep<3, double, CD_SWEEP_MERGE>
                                    : (const void*)k_sweep<3, float, CD_SWEEP_MERGE>;
    }
    if (kind == 5) {
        if (dim == 2)
            return precision == CD_FP64 ? (const void*)k_sweep<2, double, CD_SWEEP_DOMAINS>
                                        : (const void*)k_sweep<2, float, CD_SWEEP_DOMAINS>;
        return precision == CD_FP64 ? (const void*)k_sweep<3, double, CD_SWEEP_DOMAINS>
                                    : (const void*)k_sweep<3, float, CD_SWEEP_DOMAINS>;
    }
    if (kind == 4) {
        if (dim == 2)
            return precision == CD_FP64 ? (const void*)k_sweep<2, double, CD_SWEEP_MIXED>
                                        : (const void*)k_sweep<2, float, CD_SWEEP_MIXED>;
        return precision == CD_FP64 ? (const void*)k_sweep<3, double, CD_SWEEP_MIXED>
                                    : (const void*)k_sweep<3, float, CD_SWEEP_MIXED>;
    }
    if (kind == 3) {
        if (dim == 2)
            return precision == CD_FP64 ? (const void*)k_sweep_batch<2, double> : (const void*)k_sweep_batch<2, float>;
        return precision == CD_FP64 ? (const void*)k_sweep_batch<3, double> : (const void*)k_sweep_batch<3, float>;
    }
    if (dim == 2)
        return precision == CD_FP64 ? (const void*)k_sweep<2, double, CD_SWEEP_PLAIN>
                                    : (const void*)k_sweep<2, float, CD_SWEEP_PLAIN>;
    return precision == CD_FP64 ? (const void*)k_sweep<3, double, CD_SWEEP_PLAIN>
                                : (const void*)k_sweep<3, float, CD_SWEEP_PLAIN>;
}

static const int kSweepKinds[] = {0, 3, 4, 5, 6};

// Blocks of the cooperative sweep grid: one per SM (keeps the grid barrier
// cheap), for whichever of the kernels the system uses.
int cd_sweep_max_blocks(int precision, int dim, int num_sms)
{
    for (int kind : kSweepKinds) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_fn(dim, precision, kind), CD_SWEEP_THREADS, 0) !=
            cudaSuccess)
            return 0;
        if (b < 1) return 0;
    }
    return num_sms;
}

// 1 if `per_sm` blocks of `threads` threads of the sweep kernel the system
// uses can be resident on one SM.
int cd_sweep_fits(const CdGeom& g, int precision, int threads, int per_sm)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_fn(g.dim, precision, sweep_kind(g)), threads, 0) !=
        cudaSuccess)
        return 0;
    return b >= per_sm ? 1 : 0;
}

cudaError_t cd_launch_sweep(const CdGeom& g, const CdWork& w, int coop_blocks, int threads, int precision,
                            int criterion, double alpha, int max_sweeps, int pw, cudaStream_t s, int* nl)
{
    (void)pw;
    cudaError_t e = cudaMemsetAsync(w.ctrl, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    CdGeom ga = g;
    CdWork wa = w;
    int crit = criterion;
    double al = alpha;
    int ms = max_sweeps;
    void* args[] = {&ga, &wa, &crit, &al, &ms};
    const int kind = sweep_kind(g);
    ++*nl;
    return cudaLaunchCooperativeKernel(sweep_fn(g.dim, precision, kind), dim3(coop_blocks), dim3(threads),
                                       args, 0, s);
}
