// cd_adjoint.cu -- reverse-mode derivative of one CD time step (2D, FP64)
// at fixed contact states, and the tape the forward steps record for it.
//
// The paper differentiates nothing; the derivative is that of the step map
// (x, v, omega, mu) -> (x', v', omega') of Eqs. 1-2 with the converged
// impulses of the iteration (Sec. 2.1, Fig. 2, Eqs. 3-11).  Once converged,
// every contact is open (P = 0, Eq. 3), sticking (Eq. 5: the gap closes,
// u_n' = -g/dt, and there is no slip, u_t' = 0) or sliding (Eqs. 9-11:
// u_n' = -g/dt and P_t = s mu P_n).  With the states frozen these are linear
// in the impulses: S (H v' + g/dt) = 0 with v' = v_free + W H^T Phi p, where
// H maps body velocities to contact-frame relative velocities, W = diag(1/m,
// 1/m, 1/I), S keeps the rows above and Phi maps the free impulse components
// p to (P_n, P_t).  The reverse pass for an incoming gradient lambda of v'
// (plus dt times that of x', Eq. 2) solves the transposed system
//     Phi^T H Gamma = 0,   Gamma = W (lambda - H^T Y)
// for the multipliers Y by Gauss-Seidel in the same colour order as the
// forward sweep: per contact u = H Gamma, then Y += M (u_n, u_t) for a
// sticking contact, Y_n += m_n (u_n + s mu u_t) for a sliding one, and Gamma
// -= W H^T dY on the two bodies.  Then
//     dL/dv_free = lambda - H^T Y        (= dL/dv, dL/domega of the step's input)
//     dL/dmu     = sum_sliding s P_n (H Gamma)_t
//     dL/dx      = dL/dx' + sum over contacts of the derivative through the
//                  normal n and the gap g:  dL/dn = P_n dGamma + P_t R^T dGamma
//                  - Y_n dv' - Y_t R^T dv',  dL/dg = -Y_n / dt,
//                  with dGamma, dv' the differences body b - body a and
//                  R^T (u_x, u_y) = (u_y, -u_x); for a pair dn/dd = (I - n n^T)
//                  / |d|, dg/dd = n, d = x_b - x_a; for a wall dg/dx_a = -n.
// A loss that also depends on the step's wall forces (sum of the normal
// impulses on wall k over dt) adds q_n = dL/dF_k / dt to u_n on that wall's
// contacts: the rows solved become Phi^T (H Gamma + q) = 0.
// With params.adjoint_compliance eps > 0 each retained row is softened to
// Phi^T (H Gamma + q) - eps diag(w_n, w_t) Y = 0 (contacts with a small
// compliance), which makes the transposed system nonsingular on hyperstatic
// networks, where the rigid one has no unique multipliers.
// A contact whose normal impulse is at most CD_GRAZING times the step's
// largest is taken as open (two bodies left touching by an inelastic
// collision carry rounding noise there, and the map has a kink).
#include "cd_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum_a(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_a(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block sum of NV values per thread (fixed tree); valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*s_red)[4])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum_a(v[j]);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) s_red[wid][j] = v[j];
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = warp_sum_a(lane < nw ? s_red[lane][j] : 0.0);
    }
    __syncthreads();
}

// Sum (or max) over the blocks' partials, identical in every block.
template <bool MAX>
__device__ __forceinline__ double grid_reduce(const double* part, int nb, double* s_bc)
{
    if (threadIdx.x < 32) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nb; b += 32) x = MAX ? fmax(x, part[b]) : x + part[b];
        x = MAX ? warp_max_a(x) : warp_sum_a(x);
        if (threadIdx.x == 0) *s_bc = x;
    }
    __syncthreads();
    const double r = *s_bc;
    __syncthreads();
    return r;
}

__device__ __forceinline__ bool is_slide(double mu, const double2& P)
{
    return fabs(P.y) == mu * P.x;
}

// One Gauss-Seidel update of the transposed system on contact p; adds |Y|
// and |dY| to acc[0], acc[1].
__device__ __forceinline__ void adj_update(const CdGeom& g, const CdWork& w, const CdTape& t, const CdAdjIO& io,
                                           int p, double thr, double (&acc)[3])
{
    const double2 P = t.P[p];
    if (!(P.x > thr)) return;                         // open
    const int2 ab = t.ab[p];
    const bool wall = ab.y >= g.n;
    const double4_16a geo = t.geo[p];
    const double nx = geo.x, ny = geo.y, mn = geo.w, mt = t.mt[p];
    const double4_16a* S = (const double4_16a*)w.S;
    const double4_16a sa = S[ab.x];
    double4_16a Ga = w.adj_B[2 * ab.x], La = w.adj_B[2 * ab.x + 1];
    double4_16a Gb = make_double4_16a(0.0, 0.0, 0.0, 0.0), Lb = Gb, sb = Gb;
    if (!wall) {
        sb = S[ab.y];
        Gb = w.adj_B[2 * ab.y];
        Lb = w.adj_B[2 * ab.y + 1];
    }
    const double dgx = Gb.x - Ga.x, dgy = Gb.y - Ga.y;
    const double un = dgx * nx + dgy * ny + (wall ? io.wq[ab.y - g.n] : 0.0);
    const double ut = (dgy * nx - dgx * ny) - (sa.y * Ga.z + sb.y * Gb.z);
    // with compliance eps the rows are Phi^T (H Gamma + q) - eps diag(w) Y = 0
    double2 Y = w.adj_Y[p];
    const double eps = io.eps, inv1e = 1.0 / (1.0 + eps);
    double dYn, dYt;
    if (is_slide(g.mu, P)) {
        const double s = (P.y < 0.0) ? -1.0 : 1.0;
        dYn = (mn * (un + s * g.mu * ut) - eps * Y.x) * inv1e;
        dYt = 0.0;
    } else {
        dYn = (mn * un - eps * Y.x) * inv1e;
        dYt = (mt * ut - eps * Y.y) * inv1e;
    }
    const double fx = dYn * nx - dYt * ny, fy = dYn * ny + dYt * nx;
    // Gamma -= W H^T dY;  Lambda += H^T dY  (body a: -f, -r_a dY_t; body b: +f, -r_b dY_t)
    Ga.x += sa.x * fx; Ga.y += sa.x * fy; Ga.z += sa.z * dYt;
    La.x -= fx; La.y -= fy; La.z -= sa.y * dYt;
    w.adj_B[2 * ab.x] = Ga;
    w.adj_B[2 * ab.x + 1] = La;
    if (!wall) {
        Gb.x -= sb.x * fx; Gb.y -= sb.x * fy; Gb.z += sb.z * dYt;
        Lb.x += fx; Lb.y += fy; Lb.z -= sb.y * dYt;
        w.adj_B[2 * ab.y] = Gb;
        w.adj_B[2 * ab.y + 1] = Lb;
    }
    Y.x += dYn;
    Y.y += dYt;
    w.adj_Y[p] = Y;
    acc[0] += sqrt(Y.x * Y.x + Y.y * Y.y);
    acc[1] += sqrt(dYn * dYn + dYt * dYt);
}

// Position gradient through the contact's normal and gap, dL/dmu and the
// state counts; acc = (dmu, sticking, sliding).
__device__ __forceinline__ void adj_geometry(const CdGeom& g, const CdWork& w, const CdTape& t, int p, double thr,
                                             double (&acc)[3])
{
    const double2 P = t.P[p];
    if (!(P.x > thr)) return;
    const int2 ab = t.ab[p];
    const bool wall = ab.y >= g.n;
    const double4_16a geo = t.geo[p];
    const double nx = geo.x, ny = geo.y;
    const double4_16a* S = (const double4_16a*)w.S;
    const double4_16a sa = S[ab.x];
    const double4_16a Ga = w.adj_B[2 * ab.x];
    const double4_16a va = t.V[ab.x];
    double4_16a Gb = make_double4_16a(0.0, 0.0, 0.0, 0.0), vb = Gb, sb = Gb;
    if (!wall) {
        sb = S[ab.y];
        Gb = w.adj_B[2 * ab.y];
        vb = t.V[ab.y];
    } else {
        const double* u = g.wall_vel + 3 * (ab.y - g.n);
        vb.x = u[0];
        vb.y = u[1];
    }
    const double2 Y = w.adj_Y[p];
    const double dgx = Gb.x - Ga.x, dgy = Gb.y - Ga.y;
    const double dvx = vb.x - va.x, dvy = vb.y - va.y;
    if (is_slide(g.mu, P)) {
        const double s = (P.y < 0.0) ? -1.0 : 1.0;
        const double ut = (dgy * nx - dgx * ny) - (sa.y * Ga.z + sb.y * Gb.z);
        acc[0] += s * P.x * ut;
        acc[2] += 1.0;
    } else {
        acc[1] += 1.0;
    }
    w.adj_mark[ab.x] = 1;
    if (!wall) w.adj_mark[ab.y] = 1;
    const double dLg = -Y.x / g.dt;
    double2 ga = w.adj_gx[ab.x];
    if (wall) {
        ga.x -= dLg * nx;
        ga.y -= dLg * ny;
        w.adj_gx[ab.x] = ga;
        return;
    }
    const double dLnx = P.x * dgx + P.y * dgy - Y.x * dvx - Y.y * dvy;
    const double dLny = P.x * dgy - P.y * dgx - Y.x * dvy + Y.y * dvx;
    const double dist = geo.z * g.dt + sa.y + sb.y;   // |d| = g + r_a + r_b
    const double nd = nx * dLnx + ny * dLny;
    const double ddx = (dLnx - nx * nd) / dist + dLg * nx;
    const double ddy = (dLny - ny * nd) / dist + dLg * ny;
    double2 gb = w.adj_gx[ab.y];
    ga.x -= ddx; ga.y -= ddy;
    gb.x += ddx; gb.y += ddy;
    w.adj_gx[ab.x] = ga;
    w.adj_gx[ab.y] = gb;
}

__global__ void k_tape_record(CdWork w, int n, int64_t cap)
{
    const CdCtrl* ctrl = w.ctrl;
    const CdTape t = cd_tape_slot(w.tape, n, cap, ctrl->tape_slot);
    const int nc = ctrl->nc;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (tid == 0) {
        t.hdr->nc = nc;
        t.hdr->ncolours = ctrl->ncolours;
        t.hdr->valid = (ctrl->skip == 0 && ctrl->error == CDE_NONE) ? 1 : 0;
    }
    for (int k = tid; k <= CD_KMAX; k += stride) t.hdr->colour_off[k] = w.colour_off[k];
    for (int c = tid; c < nc; c += stride) {
        t.ab[c] = w.c_ab[c];
        t.geo[c] = ((const double4_16a*)w.c_geo)[c];
        t.mt[c] = ((const double*)w.c_m)[c];
        t.P[c] = ((const double2*)w.c_P)[c];
    }
    for (int i = tid; i < n; i += stride) t.V[i] = ((const double4_16a*)w.V)[i];
}

__global__ void k_tape_advance(CdCtrl* ctrl, int T)
{
    ctrl->tape_slot = (ctrl->tape_slot + 1) % T;
}

__global__ void k_set_tape_slot(CdCtrl* ctrl, int slot)
{
    ctrl->tape_slot = slot;
}

// The whole reverse step as one cooperative kernel: initial Gamma, the
// Gauss-Seidel sweeps of the transposed system (one grid barrier per colour),
// the position gradient colour by colour, then the outputs.
__global__ void __launch_bounds__(CD_SWEEP_THREADS, 1)
k_adjoint(CdGeom g, CdWork w, CdTape t, CdAdjIO io, double alpha, int max_sweeps)
{
    __shared__ int s_off[CD_KMAX + 1];
    __shared__ double s_red[CD_SWEEP_THREADS / 32][4];
    __shared__ double s_bc;
    CdCtrl* ctrl = w.ctrl;
    const int nb = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (!t.hdr->valid) {
        if (tid == 0) atomicCAS(&ctrl->error, CDE_NONE, CDE_TAPE);
        return;
    }
    const int n = g.n;
    const int nc = t.hdr->nc;
    const int K = t.hdr->ncolours;
    unsigned long long epoch = 0;
    for (int k = threadIdx.x; k <= CD_KMAX; k += blockDim.x) s_off[k] = t.hdr->colour_off[k];

    // incoming gradient: lambda = dL/dv' + dt dL/dx' (Eq. 2), Gamma = W lambda
    const double4_16a* S = (const double4_16a*)w.S;
    for (int i = tid; i < n; i += stride) {
        const double lx = io.dLv[2 * i] + g.dt * io.dLx[2 * i];
        const double ly = io.dLv[2 * i + 1] + g.dt * io.dLx[2 * i + 1];
        const double lw = io.dLw[i];
        const double im = S[i].x;
        const double iI = g.rotations ? io.inv_I[i] : 0.0;
        w.adj_B[2 * i] = make_double4_16a(im * lx, im * ly, iI * lw, 0.0);
        w.adj_B[2 * i + 1] = make_double4_16a(0.0, 0.0, 0.0, 0.0);
        w.adj_lam[i] = make_double4_16a(lx, ly, lw, 0.0);
        w.adj_gx[i] = make_double2(io.dLx[2 * i], io.dLx[2 * i + 1]);
        w.adj_mark[i] = 0;
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    // largest normal impulse (the open threshold) and the scale of the
    // multipliers the incoming gradient calls for, sum of m_n (|Gamma_a| + |Gamma_b|)
    {
        double acc[3] = {0.0, 0.0, 0.0};
        double pmax = 0.0;
        for (int c = tid; c < nc; c += stride) {
            w.adj_Y[c] = make_double2(0.0, 0.0);
            pmax = fmax(pmax, t.P[c].x);
            const int2 ab = t.ab[c];
            const double4_16a Ga = w.adj_B[2 * ab.x];
            double sc = sqrt(Ga.x * Ga.x + Ga.y * Ga.y) + S[ab.x].y * fabs(Ga.z);
            if (ab.y < n) {
                const double4_16a Gb = w.adj_B[2 * ab.y];
                sc += sqrt(Gb.x * Gb.x + Gb.y * Gb.y) + S[ab.y].y * fabs(Gb.z);
            } else {
                sc += fabs(io.wq[ab.y - n]);
            }
            acc[0] += t.geo[c].w * sc;
        }
        block_sum<3>(acc, s_red);
        pmax = warp_max_a(pmax);
        __shared__ double s_max[CD_SWEEP_THREADS / 32];
        if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = pmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, s_max[q]);
            w.partials[blockIdx.x] = m;
            w.partials[nb + blockIdx.x] = acc[0];
        }
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    const double thr = CD_GRAZING * grid_reduce<true>(w.partials, nb, &s_bc);
    const double yscale = grid_reduce<false>(w.partials + nb, nb, &s_bc);

    // sweeps until sum |dY| <= alpha max(sum |Y|, yscale)
    int sweeps = 0, converged = (nc == 0), diverged = 0;
    double resid = 0.0;
    while (!converged && sweeps < max_sweeps) {
        double* part = w.partials + (size_t)((sweeps & 1) ? 0 : 1) * 3 * nb;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < K; ++k) {
            const CdSpan sp = cd_colour_span(s_off[k], s_off[k + 1]);
            for (int p = sp.p; p < sp.end; p += blockDim.x) adj_update(g, w, t, io, p, thr, acc);
            if (k == K - 1) {
                block_sum<3>(acc, s_red);
                if (threadIdx.x == 0) {
                    part[blockIdx.x] = acc[0];
                    part[nb + blockIdx.x] = acc[1];
                }
            }
            if (!cd_grid_sync(ctrl, nb, epoch)) return;
        }
        ++sweeps;
        const double ysum = grid_reduce<false>(part, nb, &s_bc);
        const double dsum = grid_reduce<false>(part + nb, nb, &s_bc);
        const double den = fmax(ysum, yscale);
        resid = (den > 0.0) ? dsum / den : 0.0;
        converged = dsum <= alpha * den;
        if (!(ysum <= 1e30 * fmax(yscale, 1e-300))) {   // growing without bound, or not finite
            diverged = 1;
            converged = 0;
            break;
        }
    }

    // position gradient, colour by colour (a colour touches each particle once)
    double acc[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < K; ++k) {
        const CdSpan sp = cd_colour_span(s_off[k], s_off[k + 1]);
        for (int p = sp.p; p < sp.end; p += blockDim.x) adj_geometry(g, w, t, p, thr, acc);
        if (!cd_grid_sync(ctrl, nb, epoch)) return;
    }
    double acc4[4] = {acc[0], acc[1], acc[2], 0.0};
    for (int i = tid; i < n; i += stride) acc4[3] += (double)w.adj_mark[i];
    block_sum<4>(acc4, s_red);
    double* part = w.partials + (size_t)((sweeps & 1) ? 0 : 1) * 3 * nb;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = acc4[0];
        part[nb + blockIdx.x] = acc4[1];
        part[2 * nb + blockIdx.x] = acc4[2];
        // third slot of the other buffer: no sweep or scale reduction uses it
        w.partials[(size_t)((sweeps & 1) ? 1 : 0) * 3 * nb + 2 * nb + blockIdx.x] = acc4[3];
    }
    for (int i = tid; i < n; i += stride) {
        const double4_16a lam = w.adj_lam[i];
        const double4_16a L = w.adj_B[2 * i + 1];
        const double2 gx = w.adj_gx[i];
        io.ox[2 * i] = gx.x;
        io.ox[2 * i + 1] = gx.y;
        io.ov[2 * i] = lam.x - L.x;
        io.ov[2 * i + 1] = lam.y - L.y;
        io.ow[i] = lam.z - L.z;
    }
    if (!cd_grid_sync(ctrl, nb, epoch)) return;
    if (blockIdx.x == 0) {
        const double dmu = grid_reduce<false>(part, nb, &s_bc);
        const double nst = grid_reduce<false>(part + nb, nb, &s_bc);
        const double nsl = grid_reduce<false>(part + 2 * nb, nb, &s_bc);
        const double nmk = grid_reduce<false>(w.partials + (size_t)((sweeps & 1) ? 1 : 0) * 3 * nb + 2 * nb, nb, &s_bc);
        if (threadIdx.x == 0) {
            ctrl->adj_sweeps = sweeps;
            ctrl->adj_converged = converged;
            ctrl->adj_residual = resid;
            ctrl->adj_dmu = dmu;
            ctrl->adj_nc = nc;
            ctrl->adj_nstick = (long long)nst;
            ctrl->adj_nslide = (long long)nsl;
            ctrl->adj_nbodies = (long long)nmk;
            ctrl->adj_diverged = diverged;
        }
    }
}

}  // namespace

cudaError_t cd_launch_tape_record(const CdGeom& g, const CdWork& w, int64_t cap, int T, cudaStream_t s, int* nl)
{
    int blocks = (g.n + CD_BLOCK - 1) / CD_BLOCK;
    if (blocks < 64) blocks = 64;
    if (blocks > 4096) blocks = 4096;
    k_tape_record<<<blocks, CD_BLOCK, 0, s>>>(w, g.n, cap);
    k_tape_advance<<<1, 1, 0, s>>>(w.ctrl, T);
    *nl += 2;
    return cudaGetLastError();
}

cudaError_t cd_launch_set_tape_slot(const CdWork& w, int slot, cudaStream_t s, int* nl)
{
    k_set_tape_slot<<<1, 1, 0, s>>>(w.ctrl, slot);
    ++*nl;
    return cudaGetLastError();
}

int cd_adjoint_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_adjoint, CD_SWEEP_THREADS, 0) != cudaSuccess) return 0;
    return b;
}

cudaError_t cd_launch_adjoint(const CdGeom& g, const CdWork& w, const CdTape& t, const CdAdjIO& io, double alpha,
                              int max_sweeps, int coop_blocks, cudaStream_t s, int* nl)
{
    cudaError_t e = cudaMemsetAsync(w.ctrl, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    CdGeom ga = g;
    CdWork wa = w;
    CdTape ta = t;
    CdAdjIO ia = io;
    double al = alpha;
    int ms = max_sweeps;
    void* args[] = {&ga, &wa, &ta, &ia, &al, &ms};
    ++*nl;
    return cudaLaunchCooperativeKernel((const void*)k_adjoint, dim3(coop_blocks), dim3(CD_SWEEP_THREADS), args, 0, s);
}
