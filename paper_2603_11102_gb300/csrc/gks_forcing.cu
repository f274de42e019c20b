// gks_forcing.cu -- actuator-line (Sec. 3.1) and immersed-boundary (Sec. 3.2)
// body forcing, applied after the S2O4 update (end of Sec. 3.2).
//
// ALM: one block per rotor samples the velocity at every actuator point at
// t_{n+1} (trilinear, cell centres), evaluates the angle of attack, the
// synthetic polar, lift and drag (Eq. (axial-tangential)) and the axial and
// tangential forces; one warp per blade sums thrust and torque in FP64 with
// a fixed shuffle tree. A second kernel gathers, for every cell of the box
// swept by the rotor, the truncated Gaussian projection (Eq. (Gaussian)) of
// all point forces in blade-then-point order and adds dt f to the momentum.
//
// IBM: the cell fields Vbar, vbar and phi of a stationary body are computed
// once. Each step the direct-forcing iteration of Eq. (ibm-1) runs per cell
// (cells are independent for a fixed iteration count), the force sum of
// Eq. (force-ibm) is reduced in a fixed order, and the back-interpolated
// residual max_p |v_p - sum W U| is evaluated per Lagrangian point.
//
// Distances that decide the 3 eps cut are formed in FP64 with explicit
// round-to-nearest operations (no contraction), in the same order as a plain
// evaluation of sqrt(dx*dx + dy*dy + dz*dz).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "gks_bounds.cuh"
#include "gks_internal.h"

namespace gks {
namespace {

constexpr double kPi = 3.14159265358979323846;

struct Lattice {
    int n[3], P[3];
    long np;
    double x0[3], h[3];   // origin and width of the uniform lattice (a slab: its group's domain)
    int off[3];           // index of the grid's first cell in that lattice (a slab: along x)
    int prec;
};

Lattice make_lattice(const Ctx &c)
{
    Lattice L;
    for (int d = 0; d < 3; ++d) {
        L.n[d] = c.n[d];
        L.P[d] = c.P[d];
        L.x0[d] = c.x0[d];
        L.h[d] = c.hu[d];
        L.off[d] = d == 0 ? c.xoff : 0;
    }
    L.np = c.np;
    L.prec = c.prec;
    return L;
}

__device__ __forceinline__ long lin_index(const Lattice &L, int i, int j, int k)
{
    return (long)(i + G) + (long)L.P[0] * ((long)(j + G) + (long)L.P[1] * (k + G));
}

__device__ __forceinline__ double centre(const Lattice &L, int d, int i)
{
    return __dadd_rn(L.x0[d], __dmul_rn((double)(i + L.off[d]) + 0.5, L.h[d]));
}

__device__ __forceinline__ double dist(double dx, double dy, double dz)
{
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__device__ __forceinline__ void cell_state(const Lattice &L, const void *S, long lin, double q[4])
{
    if (L.prec == GKS_FP64) {
        const double *W = (const double *)S;
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v] = W[v * L.np + lin];
    } else {
        const float *W = (const float *)S;
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v] = (double)W[v * L.np + lin] + (double)W[(4 + v) * L.np + lin];
    }
}

// Trilinear interpolation of the cell-centre velocity m/rho; false when X is
// outside the hull of interior cell centres.
__device__ bool trilinear(const Lattice &L, const void *S, const double X[3], double U[3])
{
    int i0[3];
    double fr[3];
    for (int d = 0; d < 3; ++d) {
        const double s = (X[d] - L.x0[d]) / L.h[d] - 0.5 - (double)L.off[d];
        const double fl = floor(s);
        i0[d] = (int)fl;
        fr[d] = s - fl;
        if (i0[d] < 0 || i0[d] + 1 > L.n[d] - 1) {
            if (L.n[d] == 1 && s >= -0.5 && s <= 0.5) {
                i0[d] = 0;
                fr[d] = 0.0;
                continue;
            }
            return false;
        }
    }
    U[0] = U[1] = U[2] = 0.0;
    for (int c = 0; c < 8; ++c) {
        const int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        const double w = (di ? fr[0] : 1.0 - fr[0]) * (dj ? fr[1] : 1.0 - fr[1]) * (dk ? fr[2] : 1.0 - fr[2]);
        if (w == 0.0) continue;
        const int ii = L.n[0] == 1 ? 0 : i0[0] + di;
        const int jj = L.n[1] == 1 ? 0 : i0[1] + dj;
        const int kk = L.n[2] == 1 ? 0 : i0[2] + dk;
        double q[4];
        cell_state(L, S, lin_index(L, ii, jj, kk), q);
        U[0] += w * q[1] / q[0];
        U[1] += w * q[2] / q[0];
        U[2] += w * q[3] / q[0];
    }
    return true;
}

__device__ __forceinline__ double polar_cd(double a) { return 0.01 + 0.02 * a * a; }
__device__ __forceinline__ double polar_cl(double a)
{
    double c = 2.0 * kPi * sin(a);
    return c > 1.4 ? 1.4 : (c < -1.4 ? -1.4 : c);
}

// ------------------------------------------------------------------ ALM --

// Tip factor of Eq. (tip-correction): (2/pi) acos(exp(-g1 N (R - r) /
// (2 r |sin phi|))); 0 at and beyond the tip, 1 where sin phi = 0.
__device__ __forceinline__ double tip_factor(double g1, int nb, double R, double r, double phi)
{
    if (r >= R) return 0.0;
    const double x = g1 * nb * (R - r) / (2.0 * r * fabs(sin(phi)));
    return (2.0 / kPi) * acos(exp(-x));
}

__global__ void __launch_bounds__(256) alm_loads_kernel(Lattice L, const void *S, RotorDev r, Scalars *scal)
{
    const double t = scal->t + scal->dt;   // blades and samples at t_{n+1}
    const int npts = r.nb * r.np;
    for (int q = threadIdx.x; q < npts; q += blockDim.x) {
        const int b = q / r.np, p = q - b * r.np;
        const double th = r.az0 + r.omega * t + 2.0 * kPi * b / r.nb;
        const double cth = cos(th), sth = sin(th);
        const double rr = r.r[p];
        const double X[3] = {r.hub[0], r.hub[1] + rr * cth, r.hub[2] + rr * sth};
        r.X[3 * q] = X[0];
        r.X[3 * q + 1] = X[1];
        r.X[3 * q + 2] = X[2];
#pragma unroll
        for (int d = 0; d < 3; ++d) r.Xr[3 * q + d] = (float)(X[d] - r.hub[d]);
        if (p == 0) {
            r.et[2 * b] = -sth;
            r.et[2 * b + 1] = cth;
        }
        double U[3];
        double Fx = 0.0, Ft = 0.0, al = 0.0, phi = 0.0;
        if (!trilinear(L, S, X, U)) {
            atomicOr(&scal->flags, FLAG_RANGE);
        } else {
            double ux = U[0];
            double ut = -sth * U[1] + cth * U[2];
            const double wr = r.omega * rr;
            if (r.correction) {
                const double phi0 = atan2(ux, wr - ut);
                const double cd0 = polar_cd(phi0 - r.twist[p]);
                const double fac = 1.0 / (1.0 - cd0 * r.chord[p] / (4.0 * sqrt(kPi) * r.eps));
                ux *= fac;
                ut *= fac;
            }
            phi = atan2(ux, wr - ut);
            al = phi - r.twist[p];
            const double urel2 = ux * ux + (wr - ut) * (wr - ut);
            const double qd = 0.5 * r.rho_inf * r.chord[p] * r.width[p] * urel2;
            const double Lf = qd * polar_cl(al), Df = qd * polar_cd(al);
            Fx = (Lf * cos(phi) + Df * sin(phi)) * r.scale[q];
            Ft = (Lf * sin(phi) - Df * cos(phi)) * r.scale[q];
            if (r.tip) {
                Fx *= tip_factor(r.tip_g[0], r.nb, r.radius, rr, phi);
                Ft *= tip_factor(r.tip_g[1], r.nb, r.radius, rr, phi);
            }
        }
        r.F[q] = Fx;
        r.F[npts + q] = Ft;
        r.F[2 * npts + q] = al;
        r.F[3 * npts + q] = phi;
    }
    __syncthreads();
    // per-blade thrust and torque: warp b sums blade b in FP64
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < r.nb) {
        double T = 0.0, Q = 0.0;
        for (int p = lane; p < r.np; p += 32) {
            T += r.F[warp * r.np + p];
            Q += r.r[p] * r.F[npts + warp * r.np + p];
        }
        for (int o = 16; o > 0; o >>= 1) {
            T += __shfl_xor_sync(0xffffffffu, T, o);
            Q += __shfl_xor_sync(0xffffffffu, Q, o);
        }
        if (lane == 0) {
            r.out[warp] = T;
            r.out[r.nb + warp] = Q;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tt = 0.0, qq = 0.0;
        for (int b = 0; b < r.nb; ++b) {
            tt += r.out[b];
            qq += r.out[r.nb + b];
        }
        const double power = r.omega * qq;
        const double area = kPi * r.radius * r.radius;
        const double U = r.uref;
        r.out[2 * r.nb] = power;
        r.out[2 * r.nb + 1] = power / (0.5 * r.rho_inf * area * U * U * U);
        r.out[2 * r.nb + 2] = tt / (0.5 * r.rho_inf * area * U * U);
    }
}

__device__ __forceinline__ void add_comp(float &hi, float &lo, float d)
{
    const float s = hi + d;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (d - bp);
    const float l = lo + e;
    const float h2 = s + l;
    lo = l - (h2 - s);
    hi = h2;
}

// Projection of the point forces onto the cells of the rotor box (truncated
// Gaussian, Eq. (Gaussian)), blade-then-point order per cell. FP64 grids:
// distances and weights in FP64. FP32C grids: the blade screen, the
// distances and the weights in FP32 on hub-relative coordinates (error below
// 2e-6 relative in r^2); only a point whose r^2 lies within 1e-5 of the cut
// takes the FP64 distance, so that the support is decided exactly as in FP64.
template <typename R>
__global__ void __launch_bounds__(256) alm_spread_kernel(Lattice L, void *S, RotorDev r, Scalars *scal)
{
    const int bx = r.box[0][1] - r.box[0][0] + 1, by = r.box[1][1] - r.box[1][0] + 1;
    const int bz = r.box[2][1] - r.box[2][0] + 1;
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)bx * by * bz) return;
    const int i = r.box[0][0] + (int)(idx % bx);
    const int j = r.box[1][0] + (int)((idx / bx) % by);
    const int k = r.box[2][0] + (int)(idx / ((long)bx * by));
    const double xc[3] = {centre(L, 0, i), centre(L, 1, j), centre(L, 2, k)};
    const double cut = 3.0 * r.eps;
    const int npts = r.nb * r.np;
    R f[3] = {R(0), R(0), R(0)};
    bool any = false;
    if constexpr (std::is_same<R, double>::value) {
        for (int b = 0; b < r.nb; ++b) {
            const double e1 = r.et[2 * b], e2 = r.et[2 * b + 1];
            // every point of blade b lies on the segment hub + s e_r, s in
            // [rmin, rmax]; a cell farther than 3 eps from it gets nothing
            {
                const double ery = e2, erz = -e1;
                const double px = xc[0] - r.hub[0], py = xc[1] - r.hub[1], pz = xc[2] - r.hub[2];
                double sp = py * ery + pz * erz;
                sp = sp < r.rmin ? r.rmin : (sp > r.rmax ? r.rmax : sp);
                const double qy = py - sp * ery, qz = pz - sp * erz;
                if (px * px + qy * qy + qz * qz > cut * cut * (1.0 + 1e-6) + 1e-300) continue;
            }
            double fb[3] = {0.0, 0.0, 0.0};
            for (int p = 0; p < r.np; ++p) {
                const int q = b * r.np + p;
                const double rr = dist(xc[0] - r.X[3 * q], xc[1] - r.X[3 * q + 1], xc[2] - r.X[3 * q + 2]);
                if (rr > cut) continue;
                any = true;
                const double eta = exp(-(rr / r.eps) * (rr / r.eps)) * r.norm;
                const double Fx = r.F[q], Ft = r.F[npts + q];
                fb[0] += -Fx * eta;
                fb[1] += -Ft * e1 * eta;
                fb[2] += -Ft * e2 * eta;
            }
            f[0] += fb[0];
            f[1] += fb[1];
            f[2] += fb[2];
        }
    } else {
        const float pc[3] = {(float)(xc[0] - r.hub[0]), (float)(xc[1] - r.hub[1]), (float)(xc[2] - r.hub[2])};
        const float c2 = (float)(cut * cut), c2lo = c2 * (1.0f - 1e-5f), c2hi = c2 * (1.0f + 1e-5f);
        const float ie2 = (float)r.ie2, norm = (float)r.norm;
        const float rmin = (float)r.rmin, rmax = (float)r.rmax;
        for (int b = 0; b < r.nb; ++b) {
            const float e1 = (float)r.et[2 * b], e2 = (float)r.et[2 * b + 1];
            {
                float sp = pc[1] * e2 - pc[2] * e1;
                sp = fminf(fmaxf(sp, rmin), rmax);
                const float qy = pc[1] - sp * e2, qz = pc[2] + sp * e1;
                if (pc[0] * pc[0] + qy * qy + qz * qz > c2 * 1.0001f) continue;
            }
            float fb[3] = {0.0f, 0.0f, 0.0f};
            for (int p = 0; p < r.np; ++p) {
                const int q = b * r.np + p;
                const float dx = pc[0] - r.Xr[3 * q], dy = pc[1] - r.Xr[3 * q + 1], dz = pc[2] - r.Xr[3 * q + 2];
                const float s2 = dx * dx + dy * dy + dz * dz;
                if (s2 > c2hi) continue;
                if (s2 >= c2lo &&
                    dist(xc[0] - r.X[3 * q], xc[1] - r.X[3 * q + 1], xc[2] - r.X[3 * q + 2]) > cut)
                    continue;
                any = true;
                const float eta = expf(-s2 * ie2) * norm;
                const float Fx = (float)r.F[q], Ft = (float)r.F[npts + q];
                fb[0] += -Fx * eta;
                fb[1] += -Ft * e1 * eta;
                fb[2] += -Ft * e2 * eta;
            }
            f[0] += fb[0];
            f[1] += fb[1];
            f[2] += fb[2];
        }
    }
    if (!any) return;
    const long lin = lin_index(L, i, j, k);
    if (!in_bounds(lin, L.np)) return;
    const double dt = scal->dt;
    if constexpr (std::is_same<R, double>::value) {
        double *W = (double *)S;
#pragma unroll
        for (int d = 0; d < 3; ++d) W[(1 + d) * L.np + lin] += dt * f[d];
    } else {
        float *W = (float *)S;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float hi = W[(1 + d) * L.np + lin], lo = W[(5 + d) * L.np + lin];
            add_comp(hi, lo, (float)dt * f[d]);
            W[(1 + d) * L.np + lin] = hi;
            W[(5 + d) * L.np + lin] = lo;
        }
    }
}

// ------------------------------------------------------------------ IBM --

__global__ void __launch_bounds__(256) body_fields_kernel(Lattice L, BodyDev b)
{
    const int bx = b.box[0][1] - b.box[0][0] + 1, by = b.box[1][1] - b.box[1][0] + 1;
    const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= b.nbox) return;
    const int i = b.box[0][0] + (int)(c % bx);
    const int j = b.box[1][0] + (int)((c / bx) % by);
    const int k = b.box[2][0] + (int)(c / ((long)bx * by));
    const double xc[3] = {centre(L, 0, i), centre(L, 1, j), centre(L, 2, k)};
    const double vol = L.h[0] * L.h[1] * L.h[2];
    const double Delta = cbrt(vol);
    const double norm = 1.0 / (b.eps * b.eps * b.eps * pow(kPi, 1.5));
    double Vb = 0.0, vs[3] = {0.0, 0.0, 0.0};
    for (int p = 0; p < b.n; ++p) {
        const double rr = dist(xc[0] - b.xyz[3 * p], xc[1] - b.xyz[3 * p + 1], xc[2] - b.xyz[3 * p + 2]);
        if (rr > 3.0 * b.eps) continue;
        const double W = exp(-(rr / b.eps) * (rr / b.eps)) * norm * vol;
        const double Vp = Delta * b.dS[p];
        Vb += W * Vp;
        vs[0] += W * Vp * b.vel[3 * p];
        vs[1] += W * Vp * b.vel[3 * p + 1];
        vs[2] += W * Vp * b.vel[3 * p + 2];
    }
    b.Vbar[c] = Vb;
    for (int d = 0; d < 3; ++d) b.vbar[3 * c + d] = Vb > 0.0 ? vs[d] / Vb : 0.0;
    const double ph = Vb / vol;
    b.phi[c] = ph > 1.0 ? 1.0 : ph;
}

// out layout: [0..2] force on the body, [3] iterations, [4] last residual,
// [5] converged flag, [6] residual max (bits), [7..] residual per iteration
__global__ void ibm_begin_kernel(BodyDev b)
{
    for (int s = threadIdx.x; s < b.niter + 7; s += blockDim.x) b.out[s] = 0.0;
}

template <typename R>
__global__ void __launch_bounds__(256) ibm_iter_kernel(Lattice L, void *S, BodyDev b, Scalars *scal, int iters)
{
    if (b.out[5] != 0.0) return;
    const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= b.nbox) return;
    if (!(b.Vbar[c] > 0.0)) return;
    const int bx = b.box[0][1] - b.box[0][0] + 1, by = b.box[1][1] - b.box[1][0] + 1;
    const int i = b.box[0][0] + (int)(c % bx);
    const int j = b.box[1][0] + (int)((c / bx) % by);
    const int k = b.box[2][0] + (int)(c / ((long)bx * by));
    const long lin = lin_index(L, i, j, k);
    if (!in_bounds(lin, L.np)) return;
    const double dt = scal->dt;
    const double vol = L.h[0] * L.h[1] * L.h[2];
    const double phi = b.phi[c];
    if constexpr (std::is_same<R, double>::value) {
        double *W = (double *)S;
        const double rho = W[lin];
        for (int d = 0; d < 3; ++d) {
            double m = W[(1 + d) * L.np + lin];
            double fs = b.fsum[3 * c + d];
            for (int s = 0; s < iters; ++s) {
                const double U = m / rho;
                const double F = rho * phi * vol * (b.vbar[3 * c + d] - U) / dt;
                m += dt * F / vol;
                fs += F;
            }
            W[(1 + d) * L.np + lin] = m;
            b.fsum[3 * c + d] = fs;
        }
    } else {
        float *W = (float *)S;
        const float rho = W[lin] + W[4 * L.np + lin];
        const float ph = (float)phi, vo = (float)vol, dtf = (float)dt;
        for (int d = 0; d < 3; ++d) {
            float hi = W[(1 + d) * L.np + lin], lo = W[(5 + d) * L.np + lin];
            double fs = b.fsum[3 * c + d];
            for (int s = 0; s < iters; ++s) {
                const float U = (hi + lo) / rho;
                const float F = rho * ph * vo * ((float)b.vbar[3 * c + d] - U) / dtf;
                add_comp(hi, lo, dtf * F / vo);
                fs += (double)F;
            }
            W[(1 + d) * L.np + lin] = hi;
            W[(5 + d) * L.np + lin] = lo;
            b.fsum[3 * c + d] = fs;
        }
    }
}

// Cells of the box within 3 eps of point p: the clipped index cube around it.
__device__ void point_cube(const Lattice &L, const BodyDev &b, int p, int lo[3], int hi[3])
{
    const double cut = 3.0 * b.eps;
    for (int d = 0; d < 3; ++d) {
        lo[d] = (int)floor((b.xyz[3 * p + d] - cut - L.x0[d]) / L.h[d] - 0.5) - 1 - L.off[d];
        hi[d] = (int)ceil((b.xyz[3 * p + d] + cut - L.x0[d]) / L.h[d] - 0.5) + 1 - L.off[d];
        if (lo[d] < b.box[d][0]) lo[d] = b.box[d][0];
        if (hi[d] > b.box[d][1]) hi[d] = b.box[d][1];
    }
}

// Precompute of W_{ijk->p} = eta(|x_ijk - X_p|) |Omega| (Sec. 3.2): count,
// then fill in (k, j, i) order.
__global__ void __launch_bounds__(256) body_csr_kernel(Lattice L, BodyDev b, long *counts, int fill)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.n) return;
    const double vol = L.h[0] * L.h[1] * L.h[2];
    const double norm = 1.0 / (b.eps * b.eps * b.eps * pow(kPi, 1.5));
    const double cut = 3.0 * b.eps;
    const int bx = b.box[0][1] - b.box[0][0] + 1, by = b.box[1][1] - b.box[1][0] + 1;
    int lo[3], hi[3];
    point_cube(L, b, p, lo, hi);
    long o = fill ? b.csr_off[p] : 0;
    long cnt = 0;
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                const double rr = dist(centre(L, 0, i) - b.xyz[3 * p], centre(L, 1, j) - b.xyz[3 * p + 1],
                                       centre(L, 2, k) - b.xyz[3 * p + 2]);
                if (rr > cut) continue;
                if (fill) {
                    b.csr_cell[o] = (i - b.box[0][0]) + bx * ((j - b.box[1][0]) + by * (k - b.box[2][0]));
                    b.csr_w[o] = exp(-(rr / b.eps) * (rr / b.eps)) * norm * vol;
                    b.csr_wf[o] = (float)b.csr_w[o];
                    ++o;
                }
                ++cnt;
            }
    if (!fill) counts[p] = cnt;
}

// Cell velocity m/rho over the body box, input of the residual (FP64 from
// the cell state; stored as FP32 on FP32C grids).
template <typename R>
__global__ void __launch_bounds__(256) ibm_velocity_kernel(Lattice L, const void *S, BodyDev b)
{
    if (b.out[5] != 0.0) return;
    const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= b.nbox) return;
    const int bx = b.box[0][1] - b.box[0][0] + 1, by = b.box[1][1] - b.box[1][0] + 1;
    const int i = b.box[0][0] + (int)(c % bx);
    const int j = b.box[1][0] + (int)((c / bx) % by);
    const int k = b.box[2][0] + (int)(c / ((long)bx * by));
    double q[4];
    if (!in_bounds(lin_index(L, i, j, k), L.np)) return;
    cell_state(L, S, lin_index(L, i, j, k), q);
    R *U = std::is_same<R, double>::value ? (R *)b.Ubox : (R *)b.Uboxf;
#pragma unroll
    for (int d = 0; d < 3; ++d) U[3 * c + d] = (R)(q[1 + d] / q[0]);
}

// Residual max_p |v_p - sum_ijk W_{ijk->p} U_ijk|: one warp per point,
// lanes stride the point's weights, fixed shuffle tree, atomic max of the
// (non-negative) result. FP32C grids sum in FP32 (terms are ~1/nnz of |U|:
// the error stays near 1e-7 of |U|).
template <typename R>
__global__ void __launch_bounds__(256) ibm_residual_kernel(BodyDev b)
{
    if (b.out[5] != 0.0) return;
    const int warp = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= b.n) return;
    const R *Wt = std::is_same<R, double>::value ? (const R *)b.csr_w : (const R *)b.csr_wf;
    const R *U = std::is_same<R, double>::value ? (const R *)b.Ubox : (const R *)b.Uboxf;
    const long o0 = b.csr_off[warp], o1 = b.csr_off[warp + 1];
    R u0 = R(0), u1 = R(0), u2 = R(0);
    for (long o = o0 + lane; o < o1; o += 32) {
        const R W = Wt[o];
        const long c = b.csr_cell[o];
        if (!in_bounds(c, b.nbox)) continue;
        u0 += W * U[3 * c];
        u1 += W * U[3 * c + 1];
        u2 += W * U[3 * c + 2];
    }
    for (int s = 16; s > 0; s >>= 1) {
        u0 += __shfl_xor_sync(0xffffffffu, u0, s);
        u1 += __shfl_xor_sync(0xffffffffu, u1, s);
        u2 += __shfl_xor_sync(0xffffffffu, u2, s);
    }
    if (lane == 0) {
        const double e0 = b.vel[3 * warp] - (double)u0, e1 = b.vel[3 * warp + 1] - (double)u1,
                     e2 = b.vel[3 * warp + 2] - (double)u2;
        const double e = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        atomicMax((unsigned long long *)&b.out[6], (unsigned long long)__double_as_longlong(e));
    }
}

__global__ void ibm_check_kernel(BodyDev b, int s, double tol)
{
    if (b.out[5] != 0.0) return;
    const double r = __longlong_as_double(*(const long long *)&b.out[6]);
    b.out[7 + s] = r;
    b.out[4] = r;
    b.out[3] = (double)(s + 1);
    b.out[6] = 0.0;
    if (tol > 0.0 && r < tol) b.out[5] = 1.0;
}

// Force on the structure = - sum over box cells, FP64 in a fixed order:
// block k sums its contiguous chunk of cells (thread stride, then a tree)
// into part[3k..3k+2]; one block then sums the parts in order.
__global__ void __launch_bounds__(256) ibm_force_part_kernel(BodyDev b, long chunk, double *part)
{
    __shared__ double sh[3][256];
    const long c0 = blockIdx.x * chunk, c1 = min(c0 + chunk, b.nbox);
    double s[3] = {0.0, 0.0, 0.0};
    for (long c = c0 + threadIdx.x; c < c1; c += blockDim.x)
        for (int d = 0; d < 3; ++d) s[d] += b.fsum[3 * c + d];
    for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] = s[d];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[3 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) ibm_force_final_kernel(BodyDev b, const double *part, int nparts)
{
    __shared__ double sh[3][256];
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nparts; k += blockDim.x)
        for (int d = 0; d < 3; ++d) s[d] += part[3 * k + d];
    for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] = s[d];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) b.out[threadIdx.x] = -sh[threadIdx.x][0];
}

}  // namespace

void launch_alm_loads(const Ctx &c, const RotorDev &r)
{
    const Lattice L = make_lattice(c);
    alm_loads_kernel<<<1, 256, 0, c.stream>>>(L, c.state, r, c.scal);
}

void launch_alm(const Ctx &c, const RotorDev &r)
{
    const Lattice L = make_lattice(c);
    mark(c, K_ALM, 1);
    alm_loads_kernel<<<1, 256, 0, c.stream>>>(L, c.state, r, c.scal);
    mark(c, K_ALM, 0);
    launch_alm_spread(c, r);
}

void launch_alm_spread(const Ctx &c, const RotorDev &r)
{
    const Lattice L = make_lattice(c);
    const long nbox = (long)(r.box[0][1] - r.box[0][0] + 1) * (r.box[1][1] - r.box[1][0] + 1) *
                      (r.box[2][1] - r.box[2][0] + 1);
    if (nbox <= 0) return;
    const int blocks = (int)((nbox + 255) / 256);
    mark(c, K_ALM, 1);
    if (c.prec == GKS_FP64)
        alm_spread_kernel<double><<<blocks, 256, 0, c.stream>>>(L, c.state, r, c.scal);
    else
        alm_spread_kernel<float><<<blocks, 256, 0, c.stream>>>(L, c.state, r, c.scal);
    mark(c, K_ALM, 0);
}

int body_box(const Ctx &c, const double *xyz, int n, double eps, int box[3][2])
{
    const double rad = 3.0 * eps;
    for (int d = 0; d < 3; ++d) {
        double lo = INFINITY, hi = -INFINITY;
        for (int p = 0; p < n; ++p) {
            lo = fmin(lo, xyz[3 * p + d]);
            hi = fmax(hi, xyz[3 * p + d]);
        }
        const int off = d == 0 ? c.xoff : 0;
        long a = (long)floor((lo - rad - c.x0[d]) / c.hu[d] - 0.5) - 1 - off;
        long b = (long)ceil((hi + rad - c.x0[d]) / c.hu[d] - 0.5) + 1 - off;
        if (a < 0) a = 0;
        if (b > c.n[d] - 1) b = c.n[d] - 1;
        if (b < a) return -1;
        box[d][0] = (int)a;
        box[d][1] = (int)b;
    }
    return 0;
}

void launch_body_precompute(const Ctx &c, const BodyDev &b)
{
    const Lattice L = make_lattice(c);
    body_fields_kernel<<<(int)((b.nbox + 255) / 256), 256, 0, c.stream>>>(L, b);
}

void launch_body_csr_count(const Ctx &c, const BodyDev &b, long *d_counts)
{
    const Lattice L = make_lattice(c);
    body_csr_kernel<<<(b.n + 127) / 128, 128, 0, c.stream>>>(L, b, d_counts, 0);
}

void launch_body_csr_fill(const Ctx &c, const BodyDev &b)
{
    const Lattice L = make_lattice(c);
    body_csr_kernel<<<(b.n + 127) / 128, 128, 0, c.stream>>>(L, b, nullptr, 1);
}

void launch_ibm(const Ctx &c, const BodyDev &b)
{
    const Lattice L = make_lattice(c);
    const int cb = (int)((b.nbox + 255) / 256), pb = (int)(((long)b.n * 32 + 255) / 256);
    mark(c, K_IBM, 1);
    ibm_begin_kernel<<<1, 256, 0, c.stream>>>(b);
    mark(c, K_IBM, 0);
    cudaMemsetAsync(b.fsum, 0, sizeof(double) * 3 * b.nbox, c.stream);
    const int rounds = b.tol > 0.0 ? b.niter : 1;
    const int per = b.tol > 0.0 ? 1 : b.niter;
    for (int s = 0; s < rounds; ++s) {
        mark(c, K_IBM, 1);
        if (c.prec == GKS_FP64)
            ibm_iter_kernel<double><<<cb, 256, 0, c.stream>>>(L, c.state, b, c.scal, per);
        else
            ibm_iter_kernel<float><<<cb, 256, 0, c.stream>>>(L, c.state, b, c.scal, per);
        mark(c, K_IBM, 0);
        mark(c, K_IBM, 1);
        if (c.prec == GKS_FP64) {
            ibm_velocity_kernel<double><<<cb, 256, 0, c.stream>>>(L, c.state, b);
            ibm_residual_kernel<double><<<pb, 256, 0, c.stream>>>(b);
        } else {
            ibm_velocity_kernel<float><<<cb, 256, 0, c.stream>>>(L, c.state, b);
            ibm_residual_kernel<float><<<pb, 256, 0, c.stream>>>(b);
        }
        mark(c, K_IBM, 0);
        mark(c, K_IBM, 1);
        ibm_check_kernel<<<1, 1, 0, c.stream>>>(b, b.tol > 0.0 ? s : b.niter - 1, b.tol);
        mark(c, K_IBM, 0);
    }
    // the grid's reduction scratch holds kMaxPartials x 8 doubles
    const long chunk = std::max(2048L, (b.nbox + kMaxPartials - 1) / kMaxPartials);
    const int nparts = (int)((b.nbox + chunk - 1) / chunk);
    mark(c, K_IBM, 1);
    ibm_force_part_kernel<<<nparts, 256, 0, c.stream>>>(b, chunk, c.partials);
    ibm_force_final_kernel<<<1, 256, 0, c.stream>>>(b, c.partials, nparts);
    mark(c, K_IBM, 0);
}

int bounds_flag_forcing() { return bounds_flag_take(); }

}  // namespace gks
