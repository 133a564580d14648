// cd_observe.cu -- observables of the converged contact network (paper
// Sec. 4.4): the distribution of contact-force orientations (Fig. 14) and the
// stress profile across horizontal stripes (Fig. 15), computed on the device
// from the key-order contact store.
#include "cd_internal.cuh"

#define CD_PI 3.141592653589793

// phi = arctan(R_y / R_x) folded into [0, pi), counted in nbins equal bins
// (2D; contacts with a nonzero impulse).  The impulse has the force's
// direction (P = R dt).
__global__ void k_orient(CdGeom g, CdWork w, int nbins, unsigned long long* counts)
{
    const int nc = w.ctrl->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const double pn = w.Pk[2 * c], pt = w.Pk[2 * c + 1];
        if (pn == 0.0 && pt == 0.0) continue;
        const double nx = w.nrm[3 * c], ny = w.nrm[3 * c + 1];
        const double rx = __dsub_rn(__dmul_rn(pn, nx), __dmul_rn(pt, ny));
        const double ry = __dadd_rn(__dmul_rn(pn, ny), __dmul_rn(pt, nx));
        double phi = atan2(ry, rx);
        if (phi < 0.0) phi = __dadd_rn(phi, CD_PI);
        if (phi >= CD_PI) phi = __dsub_rn(phi, CD_PI);
        int bin = (int)floor(__ddiv_rn(phi, __ddiv_rn(CD_PI, (double)nbins)));
        bin = bin < 0 ? 0 : (bin >= nbins ? nbins - 1 : bin);
        atomicAdd(&counts[bin], 1ULL);
    }
}

// sum over contacts whose contact point (middle of the gap, Sec. 3.1) lies in
// stripe i of R_k l_k, with l the branch vector (centre of a to centre of b,
// or to the wall surface).  The host divides by the stripe volume.
template <int DIM>
__global__ void k_stress(CdGeom g, CdWork w, const double* __restrict__ pos, const double* __restrict__ radius,
                         int axis, double lo, double width, int ns, double* sig)
{
    const int nc = w.ctrl->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int2 ab = w.pairs[c];
        const double* n = w.nrm + 3 * c;
        double Rk;
        if (DIM == 2) {
            const double pn = w.Pk[2 * c], pt = w.Pk[2 * c + 1];
            const double tk = (axis == 0) ? -n[1] : n[0];
            Rk = (pn * n[axis] + pt * tk) / g.dt;
        } else {
            Rk = (w.Pk[4 * c] * n[axis] + w.Pk[4 * c + 1 + axis]) / g.dt;
        }
        if (Rk == 0.0) continue;
        const double ra = radius[ab.x], gap = w.gap[c];
        const double pt_k = pos[ab.x * DIM + axis] + (ra + 0.5 * gap) * n[axis];
        double lk;
        if (ab.y < g.n) {
            lk = pos[ab.y * DIM + axis] - pos[ab.x * DIM + axis];
            if (g.periodic[axis]) {
                if (lk > 0.5 * g.L[axis]) lk -= g.L[axis];
                else if (lk < -0.5 * g.L[axis]) lk += g.L[axis];
            }
        } else {
            lk = (ra + gap) * n[axis];
        }
        const double q = floor((pt_k - lo) / width);
        if (q < 0.0 || q >= (double)ns) continue;
        atomicAdd(&sig[(int)q], Rk * lk);
    }
}

cudaError_t cd_launch_orient(const CdGeom& g, const CdWork& w, int nbins, unsigned long long* counts, cudaStream_t s,
                             int* nl)
{
    int gc = (g.cap + CD_BLOCK - 1) / CD_BLOCK;
    if (gc < 1) gc = 1;
    if (gc > 4096) gc = 4096;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)nbins, s);
    if (e != cudaSuccess) return e;
    k_orient<<<gc, CD_BLOCK, 0, s>>>(g, w, nbins, counts);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t cd_launch_stress(const CdGeom& g, const CdWork& w, const double* pos, const double* radius, int axis,
                             double lo, double width, int ns, double* sig, cudaStream_t s, int* nl)
{
    int gc = (g.cap + CD_BLOCK - 1) / CD_BLOCK;
    if (gc < 1) gc = 1;
    if (gc > 4096) gc = 4096;
    cudaError_t e = cudaMemsetAsync(sig, 0, sizeof(double) * (size_t)ns, s);
    if (e != cudaSuccess) return e;
    if (g.dim == 2) k_stress<2><<<gc, CD_BLOCK, 0, s>>>(g, w, pos, radius, axis, lo, width, ns, sig);
    else k_stress<3><<<gc, CD_BLOCK, 0, s>>>(g, w, pos, radius, axis, lo, width, ns, sig);
    ++*nl;
    return cudaGetLastError();
}
