// gks_stencil.cu -- the gas-kinetic stencil of one S2O4 stage on sm_103a.
//
// Per stage and per direction d (x, y, z):
//   face_eq      one thread per tangential position of the extended face box,
//                marching 16 faces along d with a 5-cell window: WENO5-JS
//                (Sec. 2, Jiang-Shu) left/right states from one paired
//                evaluation per cell, the equilibrium state Q0 from the half
//                Maxwellians (u>0 from the left, u<0 from the right), and the
//                quartic normal slope of Q0.
//   face_flux    (x, y) persistent, face tiles loaded by TMA (32x16 with two
//                faces per thread for FP32C, 32x8 otherwise): linear quartic
//                reconstruction of Q0 and its normal slope to the 2x2 Gauss
//                points (Sec. 2, Eq. (x_example)) with the t1 pass in shared
//                memory, and the gas-kinetic flux F0 and its time derivative
//                F1 at each point (Sec. 2, Eq. (flux); Appendix), averaged
//                with weights 1/4 and stored per face. The flux of FP32 and
//                double-single arithmetic runs at two Gauss points at once on
//                packed pairs.
//   flux_update  (z) the same flux, walking z per tile column, fused with the
//                divergence (Eq. (finite)) and the two-stage fourth-order
//                combination of every cell; stage 2 also prepares the next
//                step (FP32 input, max |U|^2 for the CFL step). Double-single
//                grids store the z-face fluxes and update in update_ds_kernel.
//
// All arithmetic runs in the working type R: double for GKS_FP64, float for
// GKS_FP32C. The reconstruction works on rho - off (off = rho_ref in FP32C,
// 0 in FP64), so the large constant pressure theta * rho_ref never enters an
// FP32 difference; it cancels exactly between the two faces of a cell.
#include <cuda_runtime.h>

#include <type_traits>

#include "gks_bounds.cuh"
#include "gks_device.cuh"
#include "gks_internal.h"

namespace gks {
namespace {

using namespace dev;

// ---------------------------------------------------------------- ghosts --

template <typename R>
struct GhostArgs {
    R *w;
    long np;
    int n[3], P[3];
    int d, e1, e2, lo1, lo2, len1, len2;
    int bc0, bc1;
    R off, csound;
    R uin[3];
    int rows;   // x ghosts (d = 0): one thread per ghost of a (y, z) row, rows x 2G threads
};

template <typename R>
__global__ void __launch_bounds__(256) ghost_kernel(GhostArgs<R> A)
{
    int a, b, s, l;
    if (A.rows) {
        // x ghosts: consecutive threads take the 2G ghosts of one row, whose
        // cells are contiguous in memory (the lanes of a warp cover ~5 rows)
        const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
        const long r = t / (2 * G);
        if (r >= A.rows) return;
        const int k = (int)(t - r * 2 * G);
        s = k / G;
        l = k % G + 1;
        a = A.lo1 + (int)(r % A.len1);
        b = A.lo2 + (int)(r / A.len1);
    } else {
        a = A.lo1 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
        b = A.lo2 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
        if (a >= A.lo1 + A.len1 || b >= A.lo2 + A.len2) return;
        s = blockIdx.z / G;
        l = blockIdx.z % G + 1;
    }
    const int d = A.d, nd = A.n[d];
    const int bc = s == 0 ? A.bc0 : A.bc1;
    if (bc == GKS_BC_EXCHANGE) return;   // filled from the neighbouring slab
    const int gi = s == 0 ? -l : nd - 1 + l;
    int src;
    if (bc == GKS_BC_PERIODIC) {
        src = gi % nd;
        if (src < 0) src += nd;
    } else if (bc == GKS_BC_NOSLIP || bc == GKS_BC_SLIP) {
        src = s == 0 ? l - 1 : nd - l;
    } else {
        src = s == 0 ? 0 : nd - 1;
    }
    int cg[3], cs[3];
    cg[d] = gi; cg[A.e1] = a; cg[A.e2] = b;
    cs[d] = src; cs[A.e1] = a; cs[A.e2] = b;
    const long ig = (long)(cg[0] + G) + (long)A.P[0] * ((long)(cg[1] + G) + (long)A.P[1] * (cg[2] + G));
    const long is = (long)(cs[0] + G) + (long)A.P[0] * ((long)(cs[1] + G) + (long)A.P[1] * (cs[2] + G));
    if (!in_bounds(ig, A.np) || !in_bounds(is, A.np)) return;
    R q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = A.w[v * A.np + is];
    if (bc == GKS_BC_NOSLIP) {
        q[1] = -q[1]; q[2] = -q[2]; q[3] = -q[3];
    } else if (bc == GKS_BC_SLIP) {
        q[1 + d] = -q[1 + d];
    } else if (bc == GKS_BC_INFLOW) {
        // density from the outgoing isothermal Riemann invariant of cell 1
        const R r1 = A.off + q[0];
        const R un1 = q[1 + d] / r1;
        const R x = (s == 0 ? R(1) : R(-1)) * (A.uin[d] - un1) / A.csound;
        const R ex = exp(x);
        const R rg = r1 * ex;
        q[0] = q[0] * ex + A.off * expm1(x);   // rg - off
        q[1] = rg * A.uin[0];
        q[2] = rg * A.uin[1];
        q[3] = rg * A.uin[2];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) A.w[v * A.np + ig] = q[v];
}

template <typename R>
void ghost_impl(const Ctx &c, R *w)
{
    for (int d = 0; d < 3; ++d) {
        GhostArgs<R> A;
        A.w = w;
        A.np = c.np;
        for (int e = 0; e < 3; ++e) { A.n[e] = c.n[e]; A.P[e] = c.P[e]; }
        A.d = d;
        A.e1 = tan1(d);
        A.e2 = tan2(d);
        // axes swept before d include their ghosts (edges and corners)
        A.lo1 = A.e1 < d ? -G : 0;
        A.len1 = A.e1 < d ? c.n[A.e1] + 2 * G : c.n[A.e1];
        A.lo2 = A.e2 < d ? -G : 0;
        A.len2 = A.e2 < d ? c.n[A.e2] + 2 * G : c.n[A.e2];
        A.bc0 = c.bc[d][0];
        A.bc1 = c.bc[d][1];
        A.off = (R)c.off;
        A.csound = (R)c.csound;
        for (int e = 0; e < 3; ++e) A.uin[e] = (R)c.inflow[1 + e];
        mark(c, K_GHOST, 1);
        if (d == 0) {
            A.rows = A.len1 * A.len2;
            const long nt = (long)A.rows * 2 * G;
            ghost_kernel<R><<<(int)((nt + 255) / 256), 256, 0, c.stream>>>(A);
        } else {
            A.rows = 0;
            dim3 blk(32, 8), grd((A.len1 + 31) / 32, (A.len2 + 7) / 8, 2 * G);
            ghost_kernel<R><<<grd, blk, 0, c.stream>>>(A);
        }
        mark(c, K_GHOST, 0);
    }
}

// ------------------------------------------------------------ face state --

// Storage type of the face boxes and face fluxes between kernels: double-
// single pairs when the arithmetic is double-single (no conversion between
// the kernels), else the state's type.
template <typename R, typename C>
using Mid = typename std::conditional<std::is_same<C, dsf>::value, dsf, R>::type;

template <typename R, typename C = R>
struct FaceEqArgs {
    const R *w;      // working state, 4 arrays of np
    long np;
    Mid<R, C> *fq;   // 8 arrays of nfq
    long nfq;
    const R *ihf;    // inverse centre distance at faces of axis d
    int n1, n2;      // interior cells along t1, t2
    int e1p;         // row stride of the face box (n1 + 4 rounded up to 4)
    long sd, s1, s2; // element strides along d, t1, t2
    int cn, c1, c2;  // state component of the normal / t1 / t2 momentum
    int nf, K;       // faces along d, faces per thread of the marching kernel
    Phys<C> ph;      // in the compute type
};

// Faces per thread of the marching face-state kernels: FP32 (packed) and
// FP64 / double-single (the longer march halves the FP32 kernel's window
// warm-up at the same speed of the march itself).
constexpr int kMarch32 = 32, kMarch = 16;

// Marching variant: each thread walks K consecutive faces along d at one
// tangential position of the extended face box, with the 5 cells around the
// current cell in registers. Per cell it forms both face values of WENO5
// from one set of smoothness indicators; face f takes the right-face value
// of cell f-1 and the left-face value of cell f. Launched for FP64 grids in
// FP64 arithmetic; FP32 grids and double-single arithmetic take the packed
// variants below, which march the same way.
template <typename R, typename C = R>
__global__ void __launch_bounds__(256) face_eq_march_kernel(FaceEqArgs<R, C> A)
{
    const int a = (int)(blockIdx.x * 32 + threadIdx.x) - 2;
    const int b = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int f0 = blockIdx.z * A.K;
    if (a >= A.n1 + 2 || b >= A.n2 + 2 || f0 >= A.nf) return;
    const int f1 = min(f0 + A.K, A.nf);
    const long base = (long)(a + G) * A.s1 + (long)(b + G) * A.s2;   // cell index along d = -G
    // cells f0-3 .. f1+1 are read, faces f0 .. f1-1 written
    if (!in_bounds(base + (long)(f0 - 3 + G) * A.sd, A.np) || !in_bounds(base + (long)(f1 + 1 + G) * A.sd, A.np) ||
        !in_bounds(((long)f0 * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq) ||
        !in_bounds(((long)(f1 - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq))
        return;
    const int comp[4] = {0, A.cn, A.c1, A.c2};
    const Phys<C> &ph = A.ph;
    // window w[v][k] = cell (c - 2 + k); start with c = f0 - 1
    C w[4][5];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const R *p = A.w + comp[v] * A.np + base;
#pragma unroll
        for (int k = 0; k < 5; ++k) w[v][k] = cvt<C>(__ldg(p + (long)(f0 - 3 + k + G) * A.sd));
    }
    C Qprev[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        C l;
        weno5_pair(w[v], Qprev[v], l);
    }
    // the cell entering the window, loaded one face ahead
    R nxt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) nxt[v] = __ldg(A.w + comp[v] * A.np + base + (long)(f0 + 2 + G) * A.sd);
    for (int f = f0; f < f1; ++f) {
        C Ql[4], Qr[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
#pragma unroll
            for (int k = 0; k < 4; ++k) w[v][k] = w[v][k + 1];
            w[v][4] = cvt<C>(nxt[v]);
        }
        if (f + 1 < f1) {
            // cell f + 3 <= nf + 1 = n + 2: inside the ghost layers
#pragma unroll
            for (int v = 0; v < 4; ++v) nxt[v] = __ldg(A.w + comp[v] * A.np + base + (long)(f + 3 + G) * A.sd);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Ql[v] = Qprev[v];
            weno5_pair(w[v], Qprev[v], Qr[v]);
        }
        C Q0[4];
        face_equilibrium(ph, Ql, Qr, Q0);
        const C s = cvt<C>(A.ihf[f]) * C(1.0 / 12.0);
        const long o = ((long)f * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            A.fq[v * A.nfq + o] = cvt<Mid<R, C>>(Q0[v]);
            // cells f-2 .. f+1 are w[v][0..3]
            A.fq[(4 + v) * A.nfq + o] = cvt<Mid<R, C>>((C(15) * (w[v][2] - w[v][1]) - (w[v][3] - w[v][0])) * s);
        }
    }
}

// face_eq_march_kernel for FP32 grids on packed pairs: WENO5 of the
// components paired as (rho, m_n) and (m_t1, m_t2), the half-space terms of
// the left and right states as one pair, the normal slopes paired like the
// components. Unrolled by two so that the window shifts cost no moves.
//
// SEG (the x faces, whose cells are consecutive along the march but a row
// apart across t1): a warp's lanes are 4 consecutive march segments of K
// faces times 8 rows along t1, so that the rows a warp walks (8 per
// component instead of 32) stay in L1 for the K faces that reuse each sector;
// a store of the face box still writes 4 whole sectors (8 rows of 4
// segments).
template <bool SEG>
__global__ void __launch_bounds__(256, 3) face_eq_f2_kernel(FaceEqArgs<float, float> A)
{
    const int a = SEG ? (int)(blockIdx.x * 8 + (threadIdx.x & 7)) - 2 : (int)(blockIdx.x * 32 + threadIdx.x) - 2;
    const int b = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int f0 = SEG ? (int)(blockIdx.z * 4 + (threadIdx.x >> 3)) * A.K : (int)blockIdx.z * A.K;
    if (a >= A.n1 + 2 || b >= A.n2 + 2 || f0 >= A.nf) return;
    const int f1 = min(f0 + A.K, A.nf);
    const long base = (long)(a + G) * A.s1 + (long)(b + G) * A.s2;   // cell index along d = -G
    // cells f0-3 .. f1+1 are read, faces f0 .. f1-1 written
    if (!in_bounds(base + (long)(f0 - 3 + G) * A.sd, A.np) || !in_bounds(base + (long)(f1 + 1 + G) * A.sd, A.np) ||
        !in_bounds(((long)f0 * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq) ||
        !in_bounds(((long)(f1 - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq))
        return;
    const float *pc[4] = {A.w + base, A.w + (long)A.cn * A.np + base, A.w + (long)A.c1 * A.np + base,
                          A.w + (long)A.c2 * A.np + base};
    // window w[p][k] = cell (c - 2 + k) of component pair p; start with c = f0 - 1
    f2 w[2][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const long o = (long)(f0 - 3 + k + G) * A.sd;
#pragma unroll
        for (int q = 0; q < 2; ++q) w[q][k] = f2(__ldg(pc[2 * q] + o), __ldg(pc[2 * q + 1] + o));
    }
    f2 Qprev[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        f2 l;
        weno5_pair2(w[q], Qprev[q], l);
    }
    // the cell entering the window, loaded one face ahead
    float nxt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) nxt[v] = __ldg(pc[v] + (long)(f0 + 2 + G) * A.sd);
#pragma unroll 2
    for (int f = f0; f < f1; ++f) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
            for (int k = 0; k < 4; ++k) w[q][k] = w[q][k + 1];
            w[q][4] = f2(nxt[2 * q], nxt[2 * q + 1]);
        }
        if (f + 1 < f1) {
            // cell f + 3 <= nf + 1 = n + 2: inside the ghost layers
#pragma unroll
            for (int v = 0; v < 4; ++v) nxt[v] = __ldg(pc[v] + (long)(f + 3 + G) * A.sd);
        }
        f2 Ql[2], Qr[2], Q0[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            Ql[q] = Qprev[q];
            weno5_pair2(w[q], Qprev[q], Qr[q]);
        }
        face_equilibrium2(A.ph, Ql, Qr, Q0);
        const f2 s(A.ihf[f] * float(1.0 / 12.0));
        const long o = ((long)f * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            // cells f-2 .. f+1 are w[q][0..3]
            const f2 dq = fma(w[q][3] - w[q][0], f2(-1.0f), (w[q][2] - w[q][1]) * f2(15.0f)) * s;
            A.fq[(2 * q) * A.nfq + o] = Q0[q].v.x;
            A.fq[(2 * q + 1) * A.nfq + o] = Q0[q].v.y;
            A.fq[(4 + 2 * q) * A.nfq + o] = dq.v.x;
            A.fq[(5 + 2 * q) * A.nfq + o] = dq.v.y;
        }
    }
}

// FP32 face state of direction d: the x faces (unit stride along the
// normal) by march segments of at most 8 faces, 4 per warp.
void launch_face_eq_f2(FaceEqArgs<float, float> E, int d, cudaStream_t stream)
{
    const dim3 blk(TX, TY);
    if (d == 0 && E.sd == 1) {
        E.K = std::min(E.K, 8);
        const dim3 g((E.n1 + 4 + 7) / 8, (E.n2 + 4 + 7) / 8, (E.nf + 4 * E.K - 1) / (4 * E.K));
        face_eq_f2_kernel<true><<<g, blk, 0, stream>>>(E);
    } else {
        const dim3 g((E.n1 + 4 + 31) / 32, (E.n2 + 4 + 7) / 8, (E.nf + E.K - 1) / E.K);
        face_eq_f2_kernel<false><<<g, blk, 0, stream>>>(E);
    }
}

// face_eq_march_kernel for FP64 grids in double-single arithmetic on packed
// pairs: WENO5 of the components paired as (rho, m_n) and (m_t1, m_t2), the
// half-space terms of the left and right states as one pair, the normal
// slopes paired like the components. Every lane takes the operations of the
// scalar double-single kernel, so the face boxes have the same bits.
__global__ void __launch_bounds__(256, 2) face_eq_ds2_kernel(FaceEqArgs<double, dsf> A)
{
    const int a = (int)(blockIdx.x * 32 + threadIdx.x) - 2;
    const int b = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int f0 = blockIdx.z * A.K;
    if (a >= A.n1 + 2 || b >= A.n2 + 2 || f0 >= A.nf) return;
    const int f1 = min(f0 + A.K, A.nf);
    const long base = (long)(a + G) * A.s1 + (long)(b + G) * A.s2;   // cell index along d = -G
    // cells f0-3 .. f1+1 are read, faces f0 .. f1-1 written
    if (!in_bounds(base + (long)(f0 - 3 + G) * A.sd, A.np) || !in_bounds(base + (long)(f1 + 1 + G) * A.sd, A.np) ||
        !in_bounds(((long)f0 * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq) ||
        !in_bounds(((long)(f1 - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq))
        return;
    const double *pc[4] = {A.w + base, A.w + (long)A.cn * A.np + base, A.w + (long)A.c1 * A.np + base,
                           A.w + (long)A.c2 * A.np + base};
    // window w[p][k] = cell (c - 2 + k) of component pair p; start with c = f0 - 1
    dsf2 w[2][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const long o = (long)(f0 - 3 + k + G) * A.sd;
#pragma unroll
        for (int q = 0; q < 2; ++q) w[q][k] = dsf2(to_ds(__ldg(pc[2 * q] + o)), to_ds(__ldg(pc[2 * q + 1] + o)));
    }
    dsf2 Qprev[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        dsf2 l;
        weno5_pair(w[q], Qprev[q], l);
    }
    // the cell entering the window, loaded one face ahead
    double nxt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) nxt[v] = __ldg(pc[v] + (long)(f0 + 2 + G) * A.sd);
    for (int f = f0; f < f1; ++f) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
            for (int k = 0; k < 4; ++k) w[q][k] = w[q][k + 1];
            w[q][4] = dsf2(to_ds(nxt[2 * q]), to_ds(nxt[2 * q + 1]));
        }
        if (f + 1 < f1) {
            // cell f + 3 <= nf + 1 = n + 2: inside the ghost layers
#pragma unroll
            for (int v = 0; v < 4; ++v) nxt[v] = __ldg(pc[v] + (long)(f + 3 + G) * A.sd);
        }
        dsf Ql[4], Qr[4];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            Ql[2 * q] = Qprev[q].lane(0);
            Ql[2 * q + 1] = Qprev[q].lane(1);
            dsf2 r;
            weno5_pair(w[q], Qprev[q], r);
            Qr[2 * q] = r.lane(0);
            Qr[2 * q + 1] = r.lane(1);
        }
        dsf Q0[4];
        face_equilibrium_ds2(A.ph, Ql, Qr, Q0);
        const dsf2 s(to_ds(A.ihf[f]) * dsf(1.0 / 12.0));
        const long o = ((long)f * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            // cells f-2 .. f+1 are w[q][0..3]
            const dsf2 dq = (dsf2(15) * (w[q][2] - w[q][1]) - (w[q][3] - w[q][0])) * s;
            A.fq[(2 * q) * A.nfq + o] = Q0[2 * q];
            A.fq[(2 * q + 1) * A.nfq + o] = Q0[2 * q + 1];
            A.fq[(4 + 2 * q) * A.nfq + o] = dq.lane(0);
            A.fq[(5 + 2 * q) * A.nfq + o] = dq.lane(1);
        }
    }
}

// ------------------------------------------------------------- face flux --

template <typename R, typename C = R>
struct FluxArgs {
    Mid<R, C> *ff;   // 8 arrays of nff (0..3 F0, 4..7 F1, global components)
    long nff;
    void *gp;        // FP64 only, may be null: the 64 Gauss-point inputs per face (stride ngp)
    long ngp;
    int gp32;        // gp holds float (else double)
    const R *ih1, *ih2;  // inverse cell widths along t1, t2 (padded index)
    int n1, n2, nf;
    int gcomp[4];        // global component of local component 0..3
    Phys<C> ph;          // in the compute type
    Scalars *scal;
};

// The face average 1/4 sum of the Gauss-point fluxes in the storage type M.
template <typename M, typename C>
__device__ __forceinline__ M quarter(C acc) { return cvt<M>(acc) * M(0.25); }
template <>
__device__ __forceinline__ dsf quarter<dsf, dsf>(dsf acc) { return scale_pow2(acc, 0.25f); }

// Tile t of the face box as (t1 tile, t2 tile, face): t = ta + NA (tb + NB f).
struct TileIdx {
    int ta, tb, f;
};

// t + g for a step g given in the same mixed radix (ga < NA, gb < NB).
__device__ __forceinline__ TileIdx tile_add(TileIdx t, const TileIdx &g, int NA, int NB)
{
    t.ta += g.ta;
    t.tb += g.tb;
    t.f += g.f;
    if (t.ta >= NA) { t.ta -= NA; t.tb += 1; }
    if (t.tb >= NB) { t.tb -= NB; t.f += 1; }
    return t;
}

// t2 pass at each t1 Gauss point m, then the flux at (m, -g), (m, +g): the
// sums of F0 and F1 over the 4 Gauss points of face (tx, ty) of the tile.
// GP (the recorded steps of the adjoint) with gp set: the inputs of Gauss
// point g = 2m + n (Q0 with its density as rho, not rho - off; normal slope,
// t1 and t2 slopes; 4 components each) go to gp[(16 g + k) ngp + face], as
// double or (gp32) rounded to float (always float for R = float).
template <typename R, bool NEED_F0, bool GP = false>
__device__ __forceinline__ void tile_gauss_flux(const Phys<R> &ph, const R *st, int tx, int ty, R ih1, R ih2,
                                                R acc0[4], R acc1[4], void *gp = nullptr, int gp32 = 0,
                                                long ngp = 0, long face = 0)
{
#pragma unroll
    for (int v = 0; v < 4; ++v) acc0[v] = acc1[v] = R(0);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        R Qv[2][4], Dn[2][4], D1[2][4], D2[2][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const R *x = st + (v * 4 + m) * ST_ROWS + ty * TX + tx;
            const R *y = st + (v * 4 + 2 + m) * ST_ROWS + ty * TX + tx;
            const R *z = st + (16 + v * 2 + m) * ST_ROWS + ty * TX + tx;
            R vm, vp, dm, dp;
            tan_val_der(x[0], x[TX], x[2 * TX], x[3 * TX], x[4 * TX], vm, vp, dm, dp);
            Qv[0][v] = vm; Qv[1][v] = vp; D2[0][v] = dm; D2[1][v] = dp;
            tan_val_direct(y[0], y[TX], y[2 * TX], y[3 * TX], y[4 * TX], vm, vp);
            D1[0][v] = vm; D1[1][v] = vp;
            tan_val_direct(z[0], z[TX], z[2 * TX], z[3 * TX], z[4 * TX], vm, vp);
            Dn[0][v] = vm; Dn[1][v] = vp;
        }
        if constexpr (GP) {
          if (gp) {
#pragma unroll
            for (int nn = 0; nn < 2; ++nn) {
                const long o = (long)(16 * (2 * m + nn)) * ngp + face;
                const R q0 = Qv[nn][0] + ph.off;
                if (sizeof(R) == 8 && !gp32) {
                    R *p = (R *)gp + o;
                    p[0] = q0;
#pragma unroll
                    for (int v = 1; v < 4; ++v) p[v * ngp] = Qv[nn][v];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        p[(4 + v) * ngp] = Dn[nn][v];
                        p[(8 + v) * ngp] = D1[nn][v];
                        p[(12 + v) * ngp] = D2[nn][v];
                    }
                } else {
                    float *p = (float *)gp + o;
                    p[0] = (float)q0;
#pragma unroll
                    for (int v = 1; v < 4; ++v) p[v * ngp] = (float)Qv[nn][v];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        p[(4 + v) * ngp] = (float)Dn[nn][v];
                        p[(8 + v) * ngp] = (float)D1[nn][v];
                        p[(12 + v) * ngp] = (float)D2[nn][v];
                    }
                }
            }
          }
        }
#pragma unroll
        for (int nn = 0; nn < 2; ++nn) {
            R F0[4], F1[4];
            gk_flux<R, NEED_F0>(ph, Qv[nn], Dn[nn], D1[nn], D2[nn], ih1, ih2, F0, F1);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (NEED_F0) acc0[v] += F0[v];
                acc1[v] += F1[v];
            }
        }
    }
}

// tile_gauss_flux for FP32 arithmetic: the same t2 pass, the flux at the two
// t2 Gauss points of each t1 Gauss point as one packed evaluation.
template <bool NEED_F0>
__device__ __forceinline__ void tile_gauss_flux_f32(const Phys<float> &ph, const float *st, int tx, int ty, float ih1,
                                                    float ih2, float acc0[4], float acc1[4])
{
#pragma unroll
    for (int v = 0; v < 4; ++v) acc0[v] = acc1[v] = 0.0f;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        f2 Qv[4], Dn[4], D1[4], D2[4];   // t2 Gauss points -g, +g in the lanes
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float *x = st + (v * 4 + m) * ST_ROWS + ty * TX + tx;
            const float *y = st + (v * 4 + 2 + m) * ST_ROWS + ty * TX + tx;
            const float *z = st + (16 + v * 2 + m) * ST_ROWS + ty * TX + tx;
            tan_val_der(x[0], x[TX], x[2 * TX], x[3 * TX], x[4 * TX], Qv[v].v.x, Qv[v].v.y, D2[v].v.x, D2[v].v.y);
            tan_val_direct(y[0], y[TX], y[2 * TX], y[3 * TX], y[4 * TX], D1[v].v.x, D1[v].v.y);
            tan_val_direct(z[0], z[TX], z[2 * TX], z[3 * TX], z[4 * TX], Dn[v].v.x, Dn[v].v.y);
        }
        f2 F0[4], F1[4];
        gk_flux2<NEED_F0>(ph, Qv, Dn, D1, D2, f2(ih1), f2(ih2), F0, F1);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (NEED_F0) acc0[v] += F0[v].v.x + F0[v].v.y;
            acc1[v] += F1[v].v.x + F1[v].v.y;
        }
    }
}

// tile_gauss_flux for double-single arithmetic (no Gauss-point output): the
// same t2 pass, the flux at the two t2 Gauss points of each t1 Gauss point
// as one evaluation on packed double-single pairs, summed in the same order
// (the same bits).
template <bool NEED_F0>
__device__ __forceinline__ void tile_gauss_flux_ds2(const Phys<dsf> &ph, const Phys<dsf2> &ph2, const dsf *st, int tx,
                                                    int ty, dsf ih1, dsf ih2, dsf acc0[4], dsf acc1[4])
{
#pragma unroll
    for (int v = 0; v < 4; ++v) acc0[v] = acc1[v] = dsf(0);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        dsf2 Qv[4], Dn[4], D1[4], D2[4];   // t2 Gauss points -g, +g in the lanes
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const dsf *x = st + (v * 4 + m) * ST_ROWS + ty * TX + tx;
            const dsf *y = st + (v * 4 + 2 + m) * ST_ROWS + ty * TX + tx;
            const dsf *z = st + (16 + v * 2 + m) * ST_ROWS + ty * TX + tx;
            dsf vm, vp, dm, dp;
            tan_val_der(x[0], x[TX], x[2 * TX], x[3 * TX], x[4 * TX], vm, vp, dm, dp);
            Qv[v] = dsf2(vm, vp);
            D2[v] = dsf2(dm, dp);
            tan_val_direct(y[0], y[TX], y[2 * TX], y[3 * TX], y[4 * TX], vm, vp);
            D1[v] = dsf2(vm, vp);
            tan_val_direct(z[0], z[TX], z[2 * TX], z[3 * TX], z[4 * TX], vm, vp);
            Dn[v] = dsf2(vm, vp);
        }
        dsf2 F0[4], F1[4];
        gk_flux<dsf2, NEED_F0>(ph2, Qv, Dn, D1, D2, dsf2(ih1), dsf2(ih2), F0, F1);
#pragma unroll
        for (int nn = 0; nn < 2; ++nn)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (NEED_F0) acc0[v] += F0[v].lane(nn);
                acc1[v] += F1[v].lane(nn);
            }
    }
}

// Persistent: each block walks tiles blockIdx.x, +gridDim.x, ...; the face
// box of a tile is dead once its t1 pass is in shared memory, so the next
// tile's face box is fetched by TMA into the same buffer while the Gauss
// points of the current one are computed (one buffer: more blocks per SM).
template <typename R, typename C, bool NEED_F0, bool GP>
__global__ void __launch_bounds__(256, std::is_same<C, dsf>::value ? 2 : 1)
    face_flux_kernel(const __grid_constant__ CUtensorMap tmap, FluxArgs<R, C> A)
{
    static_assert(sizeof(C) == sizeof(R), "the t1-pass rows share the storage size");
    using M = Mid<R, C>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    M *sq = reinterpret_cast<M *>(smem_raw);             // face-box tile (SQ_N)
    C *st = reinterpret_cast<C *>(sq + SQ_N);
    uint64_t *bar = reinterpret_cast<uint64_t *>(st + ST_N);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int NA = (A.n1 + TX - 1) / TX, NB = (A.n2 + TY - 1) / TY;
    const int ntiles = NA * NB * A.nf;
    const uint32_t bytes = (uint32_t)(SQ_N * sizeof(R));
    // the block's first tile and its stride, in (ta, tb, f)
    const TileIdx g = {(int)(gridDim.x % NA), (int)((gridDim.x / NA) % NB), (int)(gridDim.x / (NA * NB))};
    TileIdx cur = {(int)(blockIdx.x % NA), (int)((blockIdx.x / NA) % NB), (int)(blockIdx.x / (NA * NB))};
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int t = blockIdx.x;
    if (tid == 0 && t < ntiles) tma_load_tile(&tmap, sq, &bar[0], cur.ta * TX, cur.tb * TY, cur.f, bytes);
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int tn = t + gridDim.x;
        const TileIdx nxt = tile_add(cur, g, NA, NB);
        const bool ok = mbar_wait(&bar[0], (uint32_t)(k & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(&A.scal->flags, FLAG_TIMEOUT);
            return;
        }
        const int a0 = cur.ta * TX, b0 = cur.tb * TY, f = cur.f;
        cur = nxt;

        tile_t1_pass(sq, st, tid);
        __syncthreads();
        // the face box is free: fetch the next tile's while this one's Gauss
        // points are computed
        if (tid == 0 && tn < ntiles) {
            fence_proxy_async();
            tma_load_tile(&tmap, sq, &bar[0], nxt.ta * TX, nxt.tb * TY, nxt.f, bytes);
        }

        const int a = a0 + tx, b = b0 + ty;
        if (a < A.n1 && b < A.n2) {
            const C ih1 = cvt<C>(__ldg(A.ih1 + a + G)), ih2 = cvt<C>(__ldg(A.ih2 + b + G));
            C acc0[4], acc1[4];
            const long o = ((long)f * A.n2 + b) * A.n1 + a;
            if constexpr (std::is_same<C, dsf>::value && !GP)
                tile_gauss_flux_ds2<NEED_F0>(A.ph, pair_phys(A.ph), st, tx, ty, ih1, ih2, acc0, acc1);
            else
                tile_gauss_flux<C, NEED_F0, GP>(A.ph, st, tx, ty, ih1, ih2, acc0, acc1, A.gp, A.gp32, A.ngp, o);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (!in_bounds(o, A.nff)) break;
                if (NEED_F0) A.ff[A.gcomp[v] * A.nff + o] = quarter<M>(acc0[v]);
                A.ff[(4 + A.gcomp[v]) * A.nff + o] = quarter<M>(acc1[v]);
            }
        }
        __syncthreads();   // st and this buffer are free again
    }
}

// The t2 pass and the flux of the two faces (tx, r0) and (tx, r0 + 1) of a
// tall tile (FP32C): each row array is read once over the 6 rows r0 .. r0+5
// that the two 5-point stencils cover; the sums of F0 and F1 over the 4
// Gauss points of each face, in the order of tile_gauss_flux.
template <bool NEED_F0>
__device__ __forceinline__ void tile_gauss_flux_pair(const Phys<float> &ph, const float *st, int tx, int r0,
                                                     float ih1, const float ih2[2], float acc0[2][4],
                                                     float acc1[2][4])
{
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc0[e][v] = acc1[e][v] = 0.0f;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        // [face][component], the two t2 Gauss points -g, +g in the lanes of a pair
        f2 Qv[2][4], Dn[2][4], D1[2][4], D2[2][4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float *x = st + (v * 4 + m) * ST_ROWS_T + r0 * TX + tx;
            const float *y = st + (v * 4 + 2 + m) * ST_ROWS_T + r0 * TX + tx;
            const float *z = st + (16 + v * 2 + m) * ST_ROWS_T + r0 * TX + tx;
            float p[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) p[i] = x[i * TX];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                tan_val_der(p[e], p[e + 1], p[e + 2], p[e + 3], p[e + 4], Qv[e][v].v.x, Qv[e][v].v.y, D2[e][v].v.x,
                            D2[e][v].v.y);
#pragma unroll
            for (int i = 0; i < 6; ++i) p[i] = y[i * TX];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                tan_val_direct(p[e], p[e + 1], p[e + 2], p[e + 3], p[e + 4], D1[e][v].v.x, D1[e][v].v.y);
#pragma unroll
            for (int i = 0; i < 6; ++i) p[i] = z[i * TX];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                tan_val_direct(p[e], p[e + 1], p[e + 2], p[e + 3], p[e + 4], Dn[e][v].v.x, Dn[e][v].v.y);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            f2 F0[4], F1[4];
            gk_flux2<NEED_F0>(ph, Qv[e], Dn[e], D1[e], D2[e], f2(ih1), f2(ih2[e]), F0, F1);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (NEED_F0) acc0[e][v] += F0[v].v.x + F0[v].v.y;
                acc1[e][v] += F1[v].v.x + F1[v].v.y;
            }
        }
    }
}

// face_flux_kernel on 32 x 16 tiles for FP32C grids (the same results bit
// for bit): the face box of a tile (its tangential halo included) arrives by
// TMA, the t1 pass fills 20 rows, and each thread computes two faces.
template <bool NEED_F0>
__global__ void __launch_bounds__(256, 2) face_flux_tall_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                FluxArgs<float, float> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *sq = reinterpret_cast<float *>(smem_raw);   // face-box tile (SQ_NT)
    float *st = sq + SQ_NT;
    uint64_t *bar = reinterpret_cast<uint64_t *>(st + ST_NT);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int NA = (A.n1 + TX - 1) / TX, NB = (A.n2 + TYT - 1) / TYT;
    const int ntiles = NA * NB * A.nf;
    const uint32_t bytes = (uint32_t)(SQ_NT * sizeof(float));
    const TileIdx g = {(int)(gridDim.x % NA), (int)((gridDim.x / NA) % NB), (int)(gridDim.x / (NA * NB))};
    TileIdx cur = {(int)(blockIdx.x % NA), (int)((blockIdx.x / NA) % NB), (int)(blockIdx.x / (NA * NB))};
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int t = blockIdx.x;
    if (tid == 0 && t < ntiles) tma_load_tile(&tmap, sq, &bar[0], cur.ta * TX, cur.tb * TYT, cur.f, bytes);
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int tn = t + gridDim.x;
        const TileIdx nxt = tile_add(cur, g, NA, NB);
        const bool ok = mbar_wait(&bar[0], (uint32_t)(k & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(&A.scal->flags, FLAG_TIMEOUT);
            return;
        }
        const int a0 = cur.ta * TX, b0 = cur.tb * TYT, f = cur.f;
        cur = nxt;

        tile_t1_pass<float, float, SQ_HT>(sq, st, tid);
        __syncthreads();
        if (tid == 0 && tn < ntiles) {
            fence_proxy_async();
            tma_load_tile(&tmap, sq, &bar[0], nxt.ta * TX, nxt.tb * TYT, nxt.f, bytes);
        }

        const int a = a0 + tx, b = b0 + 2 * ty;
        if (a < A.n1 && b < A.n2) {
            // b + 1 <= n2: inside the padded width array even when face b + 1 is not stored
            const float ih1 = __ldg(A.ih1 + a + G);
            const float ih2[2] = {__ldg(A.ih2 + b + G), __ldg(A.ih2 + b + 1 + G)};
            float acc0[2][4], acc1[2][4];
            tile_gauss_flux_pair<NEED_F0>(A.ph, st, tx, 2 * ty, ih1, ih2, acc0, acc1);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const long o = ((long)f * A.n2 + b + e) * A.n1 + a;
                if (b + e >= A.n2 || !in_bounds(o, A.nff)) break;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    if (NEED_F0) A.ff[A.gcomp[v] * A.nff + o] = acc0[e][v] * 0.25f;
                    A.ff[(4 + A.gcomp[v]) * A.nff + o] = acc1[e][v] * 0.25f;
                }
            }
        }
        __syncthreads();   // st and the face-box buffer are free again
    }
}

// ------------------------------------------------- z flux + stage update --

constexpr int kMaxPrepBoxes = 8;   // forcing boxes the fused prep can leave out



template <typename R, typename M = R>
struct UpdArgs {
    const M *ffx, *ffy;   // face fluxes of the x and y directions (8 arrays each)
    long nffx, nffy;
    const M *ffz;         // z face fluxes (the separate update of double-single FP64 grids)
    long nffz;
    const R *ihx, *ihy;   // inverse cell widths along x, y (separate update)
    const R *ihz;         // inverse cell widths along z (padded index)
    int nx, ny, nz, P0, P1;
    long np;
    const void *w0;   // stage 1: state (FP64 W / FP32C hi,lo)
    void *wk1;        // stage 1 output W* (R)
    void *pbuf;       // P
    void *state;      // stage 2 output
    R off;
    R fb[3];
    int seg;          // z-faces per segment of the fused z kernel
    // stage 2, optional: the next step's prep (FP32C: the FP32 input into
    // wk0n; max |U|^2 over the cells outside the forcing boxes into scal)
    int prep;
    float *wk0n;
    int nbox;
    int box[kMaxPrepBoxes][3][2];
};

__device__ __forceinline__ void add_comp(float &hi, float &lo, float d)
{
    // error-free two-sum of hi + d, then renormalise (hi, lo + err)
    const float s = hi + d;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (d - bp);
    const float l = lo + e;
    const float h2 = s + l;
    lo = l - (h2 - s);
    hi = h2;
}

// Stage update of one cell from the differences of its face fluxes along x,
// y, z (high minus low face, global components; entries 0..3 hold F0, used
// in stage 1 only, entries 4..7 hold F1):
//   L = -sum_d dF0_d / h_d, Lt = -sum_d dF1_d / h_d,
//   stage 1: W* = W + dt/2 L + dt^2/8 Lt, P = W + dt L + dt^2/6 Lt,
//   stage 2: W = P + dt^2/3 Lt(W*) + dt f_body.
// Returns false when a written value is not finite (stage 2).
// Double-single arithmetic on an FP64 grid: the same update with the state
// split into double-single (exact to 48 bits) and the results composed back
// into FP64.
template <int STAGE>
__device__ __forceinline__ bool update_cell_ds(const UpdArgs<double, dsf> &A, long lin, double dt, const dsf dx[],
                                               const dsf dy[], const dsf dz[], dsf ihx, dsf ihy, dsf ihz,
                                               const double s0[4], double o0[4])
{
    const dsf h = to_ds(dt), h2 = h * h;
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const dsf Lt = -(dx[4 + v] * ihx + dy[4 + v] * ihy + dz[4 + v] * ihz);
        const dsf w = to_ds(s0[v]);
        if (STAGE == 1) {
            const dsf L = -(dx[v] * ihx + dy[v] * ihy + dz[v] * ihz);
            ((double *)A.wk1)[v * A.np + lin] = to_double(w + (scale_pow2(h, 0.5f) * L + scale_pow2(h2, 0.125f) * Lt));
            ((double *)A.pbuf)[v * A.np + lin] = to_double(w + (h * L + (h2 / dsf(6.0)) * Lt));
        } else {
            dsf inc = (h2 / dsf(3.0)) * Lt;
            if (v > 0) inc += h * to_ds((double)A.fb[v - 1]);
            const double wn = to_double(w + inc);
            ((double *)A.state)[v * A.np + lin] = wn;
            bad |= !isfinite(wn);
            o0[v] = wn;
        }
    }
    return !bad;
}

template <typename R, int STAGE>
__device__ __forceinline__ bool update_cell(const UpdArgs<R> &A, long lin, double dt, const R dx[], const R dy[],
                                            const R dz[], R ihx, R ihy, R ihz, const R s0[4], const R s1[4],
                                            R o0[4], R o1[4])
{
    const R dtr = (R)dt;
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const R Lt = -(dx[4 + v] * ihx + dy[4 + v] * ihy + dz[4 + v] * ihz);
        if (STAGE == 1) {
            const R L = -(dx[v] * ihx + dy[v] * ihy + dz[v] * ihz);
            if constexpr (std::is_same<R, double>::value) {
                const double w = s0[v];
                ((double *)A.wk1)[v * A.np + lin] = w + 0.5 * dt * L + 0.125 * dt * dt * Lt;
                ((double *)A.pbuf)[v * A.np + lin] = w + dt * L + dt * dt / 6.0 * Lt;
            } else {
                float hi = s0[v], lo = s1[v];
                const float offv = v == 0 ? A.off : 0.0f;
                ((float *)A.wk1)[v * A.np + lin] = ((hi - offv) + lo) + (0.5f * dtr * L + 0.125f * dtr * dtr * Lt);
                add_comp(hi, lo, dtr * L + dtr * dtr * (1.0f / 6.0f) * Lt);
                ((float *)A.pbuf)[v * A.np + lin] = hi;
                ((float *)A.pbuf)[(4 + v) * A.np + lin] = lo;
            }
        } else {
            if constexpr (std::is_same<R, double>::value) {
                double w = s0[v] + dt * dt / 3.0 * Lt;
                if (v > 0) w += dt * (double)A.fb[v - 1];
                ((double *)A.state)[v * A.np + lin] = w;
                bad |= !isfinite(w);
                o0[v] = w;
            } else {
                float hi = s0[v], lo = s1[v];
                float inc = dtr * dtr * (1.0f / 3.0f) * Lt;
                if (v > 0) inc += dtr * A.fb[v - 1];
                add_comp(hi, lo, inc);
                ((float *)A.state)[v * A.np + lin] = hi;
                ((float *)A.state)[(4 + v) * A.np + lin] = lo;
                bad |= !isfinite(hi) || !isfinite(lo);
                o0[v] = hi;
                o1[v] = lo;
            }
        }
    }
    return !bad;
}

constexpr int SX_H = TX + 1, SX_W = TY + 1;   // x-face slab of a tile in shared memory (padded)

constexpr int SY_H = TY + 1;                  // y-face slab of a tile: the TY + 1 face rows of its cells

template <typename R>
constexpr size_t flux_update_smem_bytes(int nc)
{
    return flux_smem_bytes<R>() + (size_t)nc * (SX_H * SX_W + SY_H * TX) * sizeof(R);
}

// z-direction face flux fused with the stage update. Work items are
// (z segment, tile column) pairs, segment-major, taken round-robin by the
// persistent blocks, so that the blocks resident at one time march through
// the same z range of neighbouring columns (their tile halos and the x-face
// rows they read are shared through L2). Inside an item a block walks the
// segment's z-faces in order: F(f) - F(f-1) of the column is formed in
// registers and cell f-1 is updated at once; the first face of an item
// (the last face of the previous segment) only primes F. The x-face fluxes
// of the cell plane (x-fastest reads of a y-fastest array) and its y-face
// fluxes are copied asynchronously into shared slabs at the start of the
// tile (the x slab padded against bank conflicts), so that no register waits
// on them during the flux; the state of the thread's cell is loaded into
// registers (nothing reads it before the update).
struct ZWalk {
    int it, f, fe, f0;   // item, face, end face (exclusive), first (priming) face of the item
    int a0, b0;          // first cell of the item's tile column along x, y
};

// Item it: its segment and tile column, decoded once per item (not per face).
__device__ __forceinline__ ZWalk zwalk_item(int it, int ncol, int NA, int L, int nf)
{
    const int sgm = it / ncol, col = it - sgm * ncol, cb = col / NA;
    ZWalk z;
    z.it = it;
    z.f0 = sgm > 0 ? sgm * L - 1 : 0;
    z.f = z.f0;
    z.fe = min((sgm + 1) * L, nf);
    z.a0 = (col - cb * NA) * TX;
    z.b0 = cb * TY;
    return z;
}

template <typename R, typename C, int STAGE, bool GP>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1)
    flux_update_kernel(const __grid_constant__ CUtensorMap tmap, FluxArgs<R, C> A, UpdArgs<R, Mid<R, C>> U)
{
    static_assert(sizeof(C) == sizeof(R), "the t1-pass rows share the storage size");
    using M = Mid<R, C>;                       // face boxes, face fluxes and their differences
    // double-single grids take the z faces through face_flux_kernel and
    // update_ds_kernel instead
    static_assert(!std::is_same<C, dsf>::value, "the fused z kernel runs FP64 or FP32 arithmetic");
    constexpr bool NEED_F0 = STAGE == 1;
    constexpr int NC = STAGE == 1 ? 8 : 4, C0 = STAGE == 1 ? 0 : 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    M *sq = reinterpret_cast<M *>(smem_raw);             // face-box tile (SQ_N), refilled after its t1 pass
    C *st = reinterpret_cast<C *>(sq + SQ_N);
    uint64_t *bar = reinterpret_cast<uint64_t *>(st + ST_N);
    M *sx = reinterpret_cast<M *>(bar + 2);               // [NC][SX_H][SX_W]
    M *sy = sx + NC * SX_H * SX_W;                        // [NC][SY_H][TX]
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int NA = (A.n1 + TX - 1) / TX, NB = (A.n2 + TY - 1) / TY, nf = A.nf, L = U.seg;
    const int ncol = NA * NB, nitems = ncol * ((nf + L - 1) / L);
    if ((int)blockIdx.x >= nitems) return;
    const uint32_t bytes = (uint32_t)(SQ_N * sizeof(R));
    ZWalk cur = zwalk_item(blockIdx.x, ncol, NA, L, nf);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) tma_load_tile(&tmap, sq, &bar[0], cur.a0, cur.b0, cur.f, bytes);
    const double dt = A.scal->dt;
    bool bad = false;
    double mx = 0.0;   // stage 2 with prep: max |U|^2 of this thread's cells outside the forcing boxes
    M P0[4], P1[4];   // F0, F1 of the previous face of this column (storage type: the
                      // differences of neighbouring faces telescope exactly)
    for (int k = 0; cur.it < nitems; ++k) {
        ZWalk nxt = cur;
        if (++nxt.f >= nxt.fe) nxt = zwalk_item(cur.it + gridDim.x, ncol, NA, L, nf);
        const int f = cur.f, a0 = cur.a0, b0 = cur.b0;
        const bool upd = f > cur.f0;
        if (upd) {
            // x-face fluxes of cell plane z = f-1: faces a0 .. a0+32, rows b0 .. b0+7.
            // Thread: row y = b0 + (tid & 7), face a0 + tid/8 of every component;
            // the 8 threads with tid/8 = 0 also take face a0 + 32.
            const int yy = tid & 7, xf = tid >> 3;
            if (b0 + yy < U.ny) {
                const long sxf = (long)U.nz * U.ny;   // stride between x-faces
                const long g0 = ((long)(a0 + xf) * U.nz + (f - 1)) * U.ny + b0 + yy;
                const M *src = U.ffx + C0 * U.nffx + g0;
                if (a0 + xf <= U.nx && in_bounds(g0, U.nffx)) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) cp_async(sx + (c * SX_H + xf) * SX_W + yy, src + c * U.nffx);
                }
                if (xf == 0 && a0 + 32 <= U.nx && in_bounds(g0 + 32 * sxf, U.nffx)) {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        cp_async(sx + (c * SX_H + 32) * SX_W + yy, src + c * U.nffx + 32 * sxf);
                }
            }
            // y-face fluxes of the plane: faces b0 .. b0+8 along y, columns a0 .. a0+31.
            // Thread: column a0 + tx, face row ty of every component; face row 8 of
            // component ty.
            if (a0 + tx < U.nx) {
                const long g1 = ((long)(b0 + ty) * U.nz + (f - 1)) * U.nx + a0 + tx;
                const M *src = U.ffy + C0 * U.nffy + g1;
                if (b0 + ty <= U.ny && in_bounds(g1, U.nffy)) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) cp_async(sy + (c * SY_H + ty) * TX + tx, src + c * U.nffy);
                }
                const long g8 = g1 + (long)(TY - ty) * U.nz * U.nx;   // face row b0 + 8
                if (ty < NC && b0 + TY <= U.ny && in_bounds(g8, U.nffy))
                    cp_async(sy + (ty * SY_H + TY) * TX + tx, U.ffy + (C0 + ty) * U.nffy + g8);
            }
            cp_async_commit();
        }
        // the state of this thread's cell, loaded now so that it arrives
        // during the flux computation
        const int a = a0 + tx, b = b0 + ty;
        const bool in = a < A.n1 && b < A.n2;
        // inverse widths (x, y of the flux and the update; z of the update),
        // loaded with the prefetch so that their latency overlaps it
        R ih1 = R(0), ih2 = R(0), ihz = R(0);
        if (in) {
            ih1 = __ldg(A.ih1 + a + G);
            ih2 = __ldg(A.ih2 + b + G);
            if (upd) ihz = __ldg(U.ihz + f - 1 + G);
        }
        R s0[4], s1[4];
        long lin = 0;
        bool cell_ok = true;
        if (upd && in) {
            const int z = f - 1;
            lin = (long)(a + G) + (long)U.P0 * ((long)(b + G) + (long)U.P1 * (z + G));
            cell_ok = in_bounds(lin, U.np);
            if (cell_ok) {
                const R *src = (const R *)(STAGE == 1 ? U.w0 : U.pbuf);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    s0[v] = __ldg(src + v * U.np + lin);
                    s1[v] = std::is_same<R, double>::value ? R(0) : __ldg(src + (4 + v) * U.np + lin);
                }
            }
        }
        const bool ok = mbar_wait(&bar[0], (uint32_t)(k & 1));
        if (__syncthreads_or(!ok)) {
            cp_async_wait_all();
            if (tid == 0) atomicOr(&A.scal->flags, FLAG_TIMEOUT);
            __syncthreads();
            return;
        }
        tile_t1_pass(sq, st, tid);
        __syncthreads();
        // the face box is free: fetch the next tile's during this one's flux
        if (tid == 0 && nxt.it < nitems) {
            fence_proxy_async();
            tma_load_tile(&tmap, sq, &bar[0], nxt.a0, nxt.b0, nxt.f, bytes);
        }

        M F0[4], F1[4];
        if (in) {
            C G0[4], G1[4];
            if constexpr (std::is_same<C, float>::value && !GP)
                tile_gauss_flux_f32<NEED_F0>(A.ph, st, tx, ty, ih1, ih2, G0, G1);
            else
                tile_gauss_flux<C, NEED_F0, GP>(A.ph, st, tx, ty, cvt<C>(ih1), cvt<C>(ih2), G0, G1, A.gp, A.gp32,
                                                A.ngp, ((long)f * A.n2 + b) * A.n1 + a);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                F0[v] = NEED_F0 ? quarter<M>(G0[v]) : M(0);
                F1[v] = quarter<M>(G1[v]);
            }
        }
        if (upd) {
            cp_async_wait_all();
            __syncthreads();   // the x-face slab of every thread is in place
            if (in && cell_ok) {
                const int z = f - 1;
                M dx[8], dy[8], dz[8];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    dx[C0 + c] = sx[(c * SX_H + tx + 1) * SX_W + ty] - sx[(c * SX_H + tx) * SX_W + ty];
                    dy[C0 + c] = sy[(c * SY_H + ty + 1) * TX + tx] - sy[(c * SY_H + ty) * TX + tx];
                }
                // local frame of a z-face: (rho, m_z, m_x, m_y); global (rho, m_x, m_y, m_z)
                constexpr int loc[4] = {0, 2, 3, 1};
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    if (NEED_F0) dz[v] = F0[loc[v]] - P0[loc[v]];
                    dz[4 + v] = F1[loc[v]] - P1[loc[v]];
                }
                R o0[4], o1[4];
                bad |= !update_cell<R, STAGE>(U, lin, dt, dx, dy, dz, ih1, ih2, ihz, s0, s1, o0, o1);
                if (STAGE == 2 && U.prep) {
                    bool boxed = false;
                    for (int q = 0; q < U.nbox; ++q)
                        boxed |= a >= U.box[q][0][0] && a <= U.box[q][0][1] && b >= U.box[q][1][0] &&
                                 b <= U.box[q][1][1] && z >= U.box[q][2][0] && z <= U.box[q][2][1];
                    if constexpr (std::is_same<R, double>::value) {
                        if (!boxed) mx = max_u2(mx, cell_u2(o0));
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v) U.wk0n[v * U.np + lin] = (o0[v] - (v == 0 ? U.off : 0.0f)) + o1[v];
                        if (!boxed) mx = max_u2(mx, cell_u2(o0, o1));
                    }
                }
            }
        }
        if (in) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                P0[v] = F0[v];
                P1[v] = F1[v];
            }
        }
        cur = nxt;
        __syncthreads();   // st, the face buffer and the slabs are free again
    }
    if (STAGE == 2 && bad) atomicOr(&A.scal->flags, FLAG_NONFINITE);
    if (STAGE == 2 && U.prep) block_max_to(mx, &A.scal->maxu2_bits);
}


// Stage update of every cell from stored x, y and z face fluxes, for FP64
// grids in double-single arithmetic: there the fused z kernel needs about 220
// registers (one block per SM) while the face-flux kernel runs two blocks per
// SM, so the z faces go through face_flux_kernel into their own buffer and
// this kernel applies update_cell_ds (the same operations as the fused
// kernel, the same bits). One thread per cell of a 32 x 8 x 1 block; the
// x-face fluxes of the block's cells (y-fastest) arrive through a padded
// shared slab.
template <int STAGE>
__global__ void __launch_bounds__(256) update_ds_kernel(UpdArgs<double, dsf> U, Scalars *scal)
{
    constexpr int NC = STAGE == 1 ? 8 : 4, C0 = STAGE == 1 ? 0 : 4;
    __shared__ dsf sx[NC][SX_H][SX_W];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int a0 = blockIdx.x * TX, b0 = blockIdx.y * TY, z = blockIdx.z;
    {
        // x faces a0 .. a0+32 of rows b0 .. b0+7: thread row b0 + (tid & 7),
        // face a0 + tid/8; the 8 threads with tid/8 = 0 also take face a0 + 32
        const int yy = tid & 7, xf = tid >> 3;
        if (b0 + yy < U.ny) {
            const long sxf = (long)U.nz * U.ny;
            const long g0 = ((long)(a0 + xf) * U.nz + z) * U.ny + b0 + yy;
            if (a0 + xf <= U.nx && in_bounds(g0, U.nffx)) {
#pragma unroll
                for (int c = 0; c < NC; ++c) sx[c][xf][yy] = U.ffx[(C0 + c) * U.nffx + g0];
            }
            if (xf == 0 && a0 + 32 <= U.nx && in_bounds(g0 + 32 * sxf, U.nffx)) {
#pragma unroll
                for (int c = 0; c < NC; ++c) sx[c][32][yy] = U.ffx[(C0 + c) * U.nffx + g0 + 32 * sxf];
            }
        }
    }
    __syncthreads();
    const int a = a0 + tx, b = b0 + ty;
    bool bad = false;
    double mx = 0.0;
    if (a < U.nx && b < U.ny) {
        const long lin = (long)(a + G) + (long)U.P0 * ((long)(b + G) + (long)U.P1 * (z + G));
        const long iy = ((long)b * U.nz + z) * U.nx + a, sy = (long)U.nz * U.nx;
        const long iz = ((long)z * U.ny + b) * U.nx + a, sz = (long)U.ny * U.nx;
        if (in_bounds(lin, U.np) && in_bounds(iy + sy, U.nffy) && in_bounds(iz + sz, U.nffz)) {
            dsf dx[8], dy[8], dz[8];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int k = C0 + c;
                dx[k] = sx[c][tx + 1][ty] - sx[c][tx][ty];
                dy[k] = U.ffy[k * U.nffy + iy + sy] - U.ffy[k * U.nffy + iy];
                dz[k] = U.ffz[k * U.nffz + iz + sz] - U.ffz[k * U.nffz + iz];
            }
            const double *src = (const double *)(STAGE == 1 ? U.w0 : U.pbuf);
            double s0[4], o0[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) s0[v] = src[v * U.np + lin];
            bad = !update_cell_ds<STAGE>(U, lin, scal->dt, dx, dy, dz, to_ds(__ldg(U.ihx + a + G)),
                                         to_ds(__ldg(U.ihy + b + G)), to_ds(__ldg(U.ihz + z + G)), s0, o0);
            if (STAGE == 2 && U.prep) {
                bool boxed = false;
                for (int q = 0; q < U.nbox; ++q)
                    boxed |= a >= U.box[q][0][0] && a <= U.box[q][0][1] && b >= U.box[q][1][0] &&
                             b <= U.box[q][1][1] && z >= U.box[q][2][0] && z <= U.box[q][2][1];
                if (!boxed) mx = max_u2(mx, cell_u2(o0));
            }
        }
    }
    if (STAGE == 2 && bad) atomicOr(&scal->flags, FLAG_NONFINITE);
    if (STAGE == 2 && U.prep) block_max_to(mx, &scal->maxu2_bits);
}

// Faces per thread of the marching face-state kernel: k0 (kMarch32 or
// kMarch), halved (down to 4) while the launch would have fewer than
// min_per_sm blocks per SM, so that a smaller grid spreads its march over
// more resident blocks (each halving adds one WENO5 pair per thread to warm
// the window up). The packed FP32 kernel (3 blocks per SM) asks for 9, three
// waves: measured on 128^3, 192^3 and 384x256x256 grids this picked the
// fastest of 8, 16 and 32 faces each time (0.045, 0.122, 0.383 ms per
// launch). The FP64 kernels ask for 2.
int march_faces(long blocks_xy, int nf, int k0, int min_per_sm)
{
    int K = k0;
    while (K > 4 && blocks_xy * ((nf + K - 1) / K) < (long)min_per_sm * sm_count()) K /= 2;
    return K;
}

template <typename K>
int persistent_grid(K kernel, size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, TX * TY, smem);
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}

template <typename R, typename C, int STAGE>
struct FluxGrids {
    int flux[2] = {0, 0}, flux_update[2] = {0, 0};   // without / with the Gauss-point output
    int flux_tall = 0;                               // FP32C: 32 x 16 face tiles
};

// The Gauss-point output (recorded steps of the adjoint) exists only where the
// arithmetic type is the storage type.
template <typename R, typename C, int STAGE>
const FluxGrids<R, C, STAGE> &flux_grids()
{
    static FluxGrids<R, C, STAGE> g;
    if (!g.flux[0]) {
        constexpr size_t su = flux_update_smem_bytes<R>(STAGE == 1 ? 8 : 4);
        g.flux[0] = persistent_grid(face_flux_kernel<R, C, STAGE == 1, false>, flux_smem_bytes<R>());
        if constexpr (!std::is_same<C, dsf>::value)   // double-single: separate z update
            g.flux_update[0] = persistent_grid(flux_update_kernel<R, C, STAGE, false>, su);
        if constexpr (std::is_same<R, C>::value) {
            g.flux[1] = persistent_grid(face_flux_kernel<R, C, STAGE == 1, true>, flux_smem_bytes<R>());
            g.flux_update[1] = persistent_grid(flux_update_kernel<R, C, STAGE, true>, su);
        }
        if constexpr (std::is_same<R, float>::value && std::is_same<C, float>::value)
            g.flux_tall = persistent_grid(face_flux_tall_kernel<STAGE == 1>, flux_tall_smem_bytes());
    }
    return g;
}

// z-faces per segment of the fused z kernel: the length L that minimises the
// steps of the busiest block, ceil(items / G) x (L + 1 priming face), with
// items = columns x ceil(nf / L), over 1 to 64 segments.
int z_segment(int ncol, int nf, int G)
{
    long best = -1;
    int bestL = nf;
    for (int S = 1; S <= 64 && S <= nf; ++S) {
        const int L = (nf + S - 1) / S, Sa = (nf + L - 1) / L;
        const long items = (long)ncol * Sa;
        const long cost = (items + G - 1) / G * (L + (Sa > 1 ? 1 : 0));
        if (best < 0 || cost < best) {
            best = cost;
            bestL = L;
        }
    }
    return bestL;
}

// Arguments of the face-state kernel of direction d on working array w.
template <typename R, typename C>
FaceEqArgs<R, C> face_eq_args(const Ctx &c, int d, const R *w, const Phys<C> &ph)
{
    const long stride[3] = {1, (long)c.P[0], (long)c.P[0] * c.P[1]};
    const int t1 = tan1(d), t2 = tan2(d);
    FaceEqArgs<R, C> E;
    E.w = w;
    E.np = c.np;
    E.fq = (Mid<R, C> *)c.fq;
    E.nfq = c.nfq;
    E.ihf = (const R *)c.ihf[d];
    E.n1 = c.n[t1];
    E.n2 = c.n[t2];
    E.e1p = c.e1p[d];
    E.sd = stride[d];
    E.s1 = stride[t1];
    E.s2 = stride[t2];
    E.cn = 1 + d;
    E.c1 = 1 + t1;
    E.c2 = 1 + t2;
    E.ph = ph;
    E.nf = c.n[d] + 1;
    constexpr bool F32 = std::is_same<C, float>::value;
    E.K = march_faces((long)((E.n1 + 4 + 31) / 32) * ((E.n2 + 4 + 7) / 8), E.nf, F32 ? kMarch32 : kMarch,
                      F32 ? 9 : 2);
    return E;
}

// Arguments of the stage update of the z-face kernels (the fused one and the
// separate double-single one).
template <typename R, typename C, int STAGE>
UpdArgs<R, Mid<R, C>> update_args(const Ctx &c, const FluxArgs<R, C> &F)
{
    UpdArgs<R, Mid<R, C>> U;
    U.ffx = (const Mid<R, C> *)c.ff[0];
    U.ffy = (const Mid<R, C> *)c.ff[1];
    U.nffx = c.nff[0];
    U.nffy = c.nff[1];
    U.ffz = nullptr;
    U.nffz = 0;
    U.ihx = U.ihy = nullptr;
    U.ihz = (const R *)c.ih[2];
    U.nx = c.n[0];
    U.ny = c.n[1];
    U.nz = c.n[2];
    U.P0 = c.P[0];
    U.P1 = c.P[1];
    U.np = c.np;
    U.w0 = c.state;
    U.wk1 = c.wk1;
    U.pbuf = c.pbuf;
    U.state = c.state;
    U.off = (R)c.off;
    for (int a = 0; a < 3; ++a) U.fb[a] = (R)c.fbody[a];
    U.seg = 0;
    U.prep = STAGE == 2 && c.prep_next && c.nprep_box <= kMaxPrepBoxes;
    U.wk0n = c.prec == GKS_FP32C ? (float *)c.wk0 : nullptr;
    U.nbox = U.prep ? c.nprep_box : 0;
    for (int q = 0; q < U.nbox; ++q)
        for (int e = 0; e < 3; ++e)
            for (int k = 0; k < 2; ++k) U.box[q][e][k] = c.prep_box[q][e][k];
    return U;
}

template <typename R, typename C, int STAGE>
void stage_impl(const Ctx &c)
{
    const Phys<C> ph = make_phys<C>(c);
    const R *w = (const R *)(STAGE == 1 ? c.wk0 : c.wk1);
    const FluxGrids<R, C, STAGE> &grids = flux_grids<R, C, STAGE>();
    const dim3 blk(TX, TY);
    for (int d = 0; d < 3; ++d) {
        const int t1 = tan1(d), t2 = tan2(d);
        const FaceEqArgs<R, C> E = face_eq_args<R, C>(c, d, w, ph);
        const CUtensorMap &tmap = c.tmap[d];
        dim3 ge((E.n1 + 4 + 31) / 32, (E.n2 + 4 + 7) / 8, (E.nf + E.K - 1) / E.K);
        mark(c, K_FACE_EQ, 1);
        if constexpr (std::is_same<C, dsf>::value)
            face_eq_ds2_kernel<<<ge, blk, 0, c.stream>>>(E);
        else if constexpr (std::is_same<C, float>::value)
            launch_face_eq_f2(E, d, c.stream);
        else
            face_eq_march_kernel<R, C><<<ge, blk, 0, c.stream>>>(E);
        mark(c, K_FACE_EQ, 0);

        FluxArgs<R, C> F;
        F.ff = (Mid<R, C> *)c.ff[d];
        F.nff = c.nff[d];
        F.ih1 = (const R *)c.ih[t1];
        F.ih2 = (const R *)c.ih[t2];
        F.n1 = c.n[t1];
        F.n2 = c.n[t2];
        F.nf = c.n[d] + 1;
        F.gcomp[0] = 0;
        F.gcomp[1] = 1 + d;
        F.gcomp[2] = 1 + t1;
        F.gcomp[3] = 1 + t2;
        F.ph = ph;
        F.scal = c.scal;
        F.gp = c.gp_dir[d];
        F.ngp = c.ngp;
        F.gp32 = c.gp_bytes == 4;
        const long ntiles = (long)((F.n1 + TX - 1) / TX) * ((F.n2 + TY - 1) / TY) * F.nf;
        const int grp = d < 2 ? K_FACE_FLUX : K_FLUX_UPDATE;
        mark(c, grp, 1);
        const int gpo = F.gp != nullptr;
        if constexpr (!std::is_same<R, C>::value) F.gp = nullptr;
        if constexpr (std::is_same<C, dsf>::value) {
            if (d == 2) {
                // double-single: z-face fluxes into their own buffer, then the update
                const int grid = (int)(ntiles < grids.flux[0] ? ntiles : grids.flux[0]);
                face_flux_kernel<R, C, STAGE == 1, false><<<grid, blk, flux_smem_bytes<R>(), c.stream>>>(tmap, F);
                UpdArgs<R, Mid<R, C>> U = update_args<R, C, STAGE>(c, F);
                U.ffz = (const Mid<R, C> *)c.ff[2];
                U.nffz = c.nff[2];
                U.ihx = (const R *)c.ih[0];
                U.ihy = (const R *)c.ih[1];
                const dim3 gu((c.n[0] + TX - 1) / TX, (c.n[1] + TY - 1) / TY, c.n[2]);
                update_ds_kernel<STAGE><<<gu, blk, 0, c.stream>>>(U, c.scal);
                mark(c, grp, 0);
                continue;
            }
        }
        if (d < 2) {
            const int grid = (int)(ntiles < grids.flux[gpo] ? ntiles : grids.flux[gpo]);
            if constexpr (std::is_same<R, float>::value && std::is_same<C, float>::value) {
                if (!gpo) {
                    const long nt = (long)((F.n1 + TX - 1) / TX) * ((F.n2 + TYT - 1) / TYT) * F.nf;
                    const int gt = (int)(nt < grids.flux_tall ? nt : grids.flux_tall);
                    face_flux_tall_kernel<STAGE == 1><<<gt, blk, flux_tall_smem_bytes(), c.stream>>>(c.tmapT[d], F);
                    mark(c, grp, 0);
                    continue;
                }
            }
            if constexpr (std::is_same<R, C>::value) {
                if (gpo)
                    face_flux_kernel<R, C, STAGE == 1, true><<<grid, blk, flux_smem_bytes<R>(), c.stream>>>(tmap, F);
                else
                    face_flux_kernel<R, C, STAGE == 1, false><<<grid, blk, flux_smem_bytes<R>(), c.stream>>>(tmap, F);
            } else {
                face_flux_kernel<R, C, STAGE == 1, false><<<grid, blk, flux_smem_bytes<R>(), c.stream>>>(tmap, F);
            }
        } else {
            // z faces: flux and the stage update of every cell
            UpdArgs<R, Mid<R, C>> U = update_args<R, C, STAGE>(c, F);
            const int ncol = ((F.n1 + TX - 1) / TX) * ((F.n2 + TY - 1) / TY);
            U.seg = z_segment(ncol, F.nf, grids.flux_update[gpo]);
            const long nitems = (long)ncol * ((F.nf + U.seg - 1) / U.seg);
            const int grid = (int)(nitems < grids.flux_update[gpo] ? nitems : grids.flux_update[gpo]);
            constexpr size_t su = flux_update_smem_bytes<R>(STAGE == 1 ? 8 : 4);
            if constexpr (std::is_same<R, C>::value) {
                if (gpo)
                    flux_update_kernel<R, C, STAGE, true><<<grid, blk, su, c.stream>>>(tmap, F, U);
                else
                    flux_update_kernel<R, C, STAGE, false><<<grid, blk, su, c.stream>>>(tmap, F, U);
            }
        }
        mark(c, grp, 0);
    }
}

// ----------------------------------------------------- prep, CFL, misc --

constexpr int kPrepZ = 8;   // z planes per block of the prep / CFL kernel

// Start of a step: the largest |U|^2 over the interior cells (for the CFL
// time step) and, for FP32C, the FP32 reconstruction input hi + lo (density
// as rho - off), over the interior cells [lo, hi) of a box (the whole
// interior, or a forcing box after the forcing). One atomicMax per block.
template <int PREC>
__global__ void __launch_bounds__(256) prep_cfl_kernel(const void *__restrict__ S, float *__restrict__ wk, long np,
                                                       int3 lo, int3 hi, int P0, int P1, float off, Scalars *scal)
{
    const int i = lo.x + blockIdx.x * 32 + threadIdx.x, j = lo.y + blockIdx.y * 8 + threadIdx.y;
    const int k0 = lo.z + blockIdx.z * kPrepZ, k1 = min(k0 + kPrepZ, hi.z);
    double mx = 0.0;
    if (i < hi.x && j < hi.y) {
        for (int k = k0; k < k1; ++k) {
            const long lin = (long)(i + G) + (long)P0 * ((long)(j + G) + (long)P1 * (k + G));
            if (PREC == GKS_FP64) {
                const double *__restrict__ W = (const double *)S;
                double w[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) w[v] = W[v * np + lin];
                mx = max_u2(mx, cell_u2(w));
            } else {
                const float *__restrict__ W = (const float *)S;
                float h[4], l[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    h[v] = W[v * np + lin];
                    l[v] = W[(4 + v) * np + lin];
                }
#pragma unroll
                for (int v = 0; v < 4; ++v) wk[v * np + lin] = (h[v] - (v == 0 ? off : 0.0f)) + l[v];
                mx = max_u2(mx, cell_u2(h, l));
            }
        }
    }
    block_max_to(mx, &scal->maxu2_bits);
}

__device__ __forceinline__ void load_cell(int prec, const void *S, long np, long lin, double q[4])
{
    if (prec == GKS_FP64) {
        const double *W = (const double *)S;
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v] = W[v * np + lin];
    } else {
        const float *W = (const float *)S;
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v] = (double)W[v * np + lin] + (double)W[(4 + v) * np + lin];
    }
}

__global__ void dt_kernel(Scalars *scal, double cfl, double dt_fixed, double hmin, double csound)
{
    const double umax = sqrt(__longlong_as_double((long long)scal->maxu2_bits));
    double dt;
    if (dt_fixed > 0.0) {
        dt = dt_fixed;
        const double num = dt * (umax + csound) / hmin;
        scal->cfl_number = num;
        if (cfl > 0.0 && !(num <= cfl)) atomicOr(&scal->flags, FLAG_CFL);
    } else {
        dt = cfl * hmin / (umax + csound);
        scal->cfl_number = cfl;
        if (!isfinite(dt)) atomicOr(&scal->flags, FLAG_NONFINITE);
    }
    scal->dt = dt;
    scal->maxu2_bits = 0ull;
}

__global__ void advance_kernel(Scalars *scal) { scal->t = scal->t + scal->dt; }


// Compact FP64 state -> the padded state (FP32C: hi = fl32(q), lo =
// fl32(q - hi)), kPrepZ planes per block. With scal set it also does the
// work of prep_cfl on the new state (FP32 input into wk for FP32C, max
// |U|^2 into scal; FP32C takes the max over the FP32 values of cell_u2,
// whose order and NaN the conversion to double keeps).
__global__ void __launch_bounds__(256) scatter_kernel(int prec, const double *__restrict__ src, void *S, long np,
                                                      int nx, int ny, int nz, int P0, int P1, float *wk, float off,
                                                      Scalars *scal)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int k0 = blockIdx.z * kPrepZ, k1 = min(k0 + kPrepZ, nz);
    const long N = (long)nx * ny * nz;
    double mx = 0.0;
    float mxf = 0.0f;
    if (i < nx && j < ny) {
        // the next plane's values are loaded while this one's are stored
        double qn[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) qn[v] = k0 < k1 ? src[v * N + i + (long)nx * (j + (long)ny * k0)] : 0.0;
        for (int k = k0; k < k1; ++k) {
            const long lin = (long)(i + G) + (long)P0 * ((long)(j + G) + (long)P1 * (k + G));
            double q[4];
            float h[4], l[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) q[v] = qn[v];
            if (k + 1 < k1) {
                const long cn = i + (long)nx * (j + (long)ny * (k + 1));
#pragma unroll
                for (int v = 0; v < 4; ++v) qn[v] = src[v * N + cn];
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                if (prec == GKS_FP64) {
                    ((double *)S)[v * np + lin] = q[v];
                } else {
                    split_hi_lo(q[v], h[v], l[v]);
                    ((float *)S)[v * np + lin] = h[v];
                    ((float *)S)[(4 + v) * np + lin] = l[v];
                }
            }
            if (scal) {
                if (prec == GKS_FP64) {
                    mx = max_u2(mx, cell_u2(q));
                } else {
#pragma unroll
                    for (int v = 0; v < 4; ++v) wk[v * np + lin] = (h[v] - (v == 0 ? off : 0.0f)) + l[v];
                    mxf = max_u2f(mxf, cell_u2f(h, l));
                }
            }
        }
    }
    if (scal) block_max_to(prec == GKS_FP64 ? mx : (double)mxf, &scal->maxu2_bits);
}

__global__ void __launch_bounds__(256) gather_kernel(int prec, const void *S, double *dst, long np,
                                                     int nx, int ny, int nz, int P0, int P1)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long N = (long)nx * ny * nz;
    const long ci = i + (long)nx * (j + (long)ny * k);
    const long lin = (long)(i + G) + (long)P0 * ((long)(j + G) + (long)P1 * (k + G));
    double q[4];
    load_cell(prec, S, np, lin, q);
#pragma unroll
    for (int v = 0; v < 4; ++v) dst[v * N + ci] = q[v];
}

// FP64 sums of mass, momentum and kinetic energy: per-block partial sums in
// a fixed order, then one block adds the partials in order (deterministic).
__global__ void __launch_bounds__(256) diag_partial_kernel(int prec, const void *S, long np, int nx,
                                                           int ny, int nz, int P0, int P1,
                                                           const double *hx, const double *hy,
                                                           const double *hz, double *partials)
{
    __shared__ double sh[5][256];
    const long ncell = (long)nx * ny * nz;
    double s[5] = {0, 0, 0, 0, 0};
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
         c += (long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const long r = c / nx;
        const int j = (int)(r % ny), k = (int)(r / ny);
        const long lin = (long)(i + G) + (long)P0 * ((long)(j + G) + (long)P1 * (k + G));
        double q[4];
        load_cell(prec, S, np, lin, q);
        const double vol = hx[i + G] * hy[j + G] * hz[k + G];
        s[0] += q[0] * vol;
        s[1] += q[1] * vol;
        s[2] += q[2] * vol;
        s[3] += q[3] * vol;
        s[4] += 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0] * vol;
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) partials[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) diag_final_kernel(const double *partials, int nparts, double *out)
{
    __shared__ double sh[5][256];
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] += partials[b * 8 + q];
#pragma unroll
    for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) fill_rest_kernel(int prec, void *S, long np, int nx, int ny,
                                                        int nz, int P0, int P1)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long lin = (long)(i + G) + (long)P0 * ((long)(j + G) + (long)P1 * (k + G));
    if (prec == GKS_FP64)
        ((double *)S)[lin] = 1.0;
    else
        ((float *)S)[lin] = 1.0f;
}

// Copy the stored component arrays (4 doubles or 8 floats per cell) between
// the padded state and a compact interior array (x fastest).
template <typename T>
__global__ void __launch_bounds__(256) raw_copy_kernel(T *S, T *cpt, int narr, long np, int nx, int ny,
                                                       int nz, int P0, int P1, int to_compact)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long N = (long)nx * ny * nz;
    const long ci = i + (long)nx * (j + (long)ny * k);
    const long lin = (long)(i + G) + (long)P0 * ((long)(j + G) + (long)P1 * (k + G));
    for (int a = 0; a < narr; ++a) {
        if (to_compact)
            cpt[a * N + ci] = S[a * np + lin];
        else
            S[a * np + lin] = cpt[a * N + ci];
    }
}

int reduce_blocks(long ncell)
{
    long b = (ncell + 255) / 256;
    if (b > kMaxPartials) b = kMaxPartials;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

void launch_prep_box(const Ctx &c, const int box[3][2])
{
    const int3 lo = make_int3(box[0][0], box[1][0], box[2][0]);
    const int3 hi = make_int3(box[0][1] + 1, box[1][1] + 1, box[2][1] + 1);
    if (hi.x <= lo.x || hi.y <= lo.y || hi.z <= lo.z) return;
    dim3 blk(32, 8), g((hi.x - lo.x + 31) / 32, (hi.y - lo.y + 7) / 8, (hi.z - lo.z + kPrepZ - 1) / kPrepZ);
    const int grp = c.prec == GKS_FP32C ? K_PREP : K_CFL;
    mark(c, grp, 1);
    if (c.prec == GKS_FP32C)
        prep_cfl_kernel<GKS_FP32C><<<g, blk, 0, c.stream>>>(c.state, (float *)c.wk0, c.np, lo, hi, c.P[0], c.P[1],
                                                           (float)c.off, c.scal);
    else
        prep_cfl_kernel<GKS_FP64><<<g, blk, 0, c.stream>>>(c.state, nullptr, c.np, lo, hi, c.P[0], c.P[1], 0.0f,
                                                          c.scal);
    mark(c, grp, 0);
}

void launch_prep(const Ctx &c)
{
    const int box[3][2] = {{0, c.n[0] - 1}, {0, c.n[1] - 1}, {0, c.n[2] - 1}};
    launch_prep_box(c, box);
}

void launch_ghost(const Ctx &c, void *w)
{
    if (c.prec == GKS_FP64)
        ghost_impl<double>(c, (double *)w);
    else
        ghost_impl<float>(c, (float *)w);
}

// ------------------------------------------------------------ slab groups --

// One thread per element of the G x-planes: (component, row, plane) with
// row = the (y, z) position over the padded P1 x P2 rows.
template <typename T>
__global__ void __launch_bounds__(256) halo_copy_kernel(const T *__restrict__ src, long np_src, int P0_src, int i_src,
                                                        T *__restrict__ dst, long np_dst, int P0_dst, int i_dst,
                                                        long rows)
{
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long per = rows * G;
    if (t >= 4 * per) return;
    const int v = (int)(t / per);
    const long r = t - v * per, row = r / G;
    const int l = (int)(r - row * G);
    const long is = (long)(i_src + l) + (long)P0_src * row, id = (long)(i_dst + l) + (long)P0_dst * row;
    if (!in_bounds(is, np_src) || !in_bounds(id, np_dst)) return;
    dst[v * np_dst + id] = src[v * np_src + is];
}

void launch_halo_copy(const Ctx &src, const void *w_src, int side_src, const Ctx &dst, void *w_dst, int side_dst)
{
    // padded x index of the first plane: the interior planes next to the
    // low side start at G, next to the high side at n; the ghost planes of
    // the low side start at 0, of the high side at n + G
    const int i_src = side_src == 0 ? G : src.n[0];
    const int i_dst = side_dst == 0 ? 0 : dst.n[0] + G;
    const long rows = (long)src.P[1] * src.P[2];
    const long nt = 4 * rows * G;
    const int grid = (int)((nt + 255) / 256);
    mark(dst, K_GHOST, 1);
    if (src.prec == GKS_FP64)
        halo_copy_kernel<double><<<grid, 256, 0, dst.stream>>>((const double *)w_src, src.np, src.P[0], i_src,
                                                                (double *)w_dst, dst.np, dst.P[0], i_dst, rows);
    else
        halo_copy_kernel<float><<<grid, 256, 0, dst.stream>>>((const float *)w_src, src.np, src.P[0], i_src,
                                                               (float *)w_dst, dst.np, dst.P[0], i_dst, rows);
    mark(dst, K_GHOST, 0);
}

struct GroupScal {
    Scalars *p[64];
};

__global__ void group_max_u2_kernel(GroupScal g, int n)
{
    unsigned long long m = 0ull;   // bits of non-negative doubles order like the values
    for (int s = 0; s < n; ++s) m = max(m, g.p[s]->maxu2_bits);
    for (int s = 0; s < n; ++s) g.p[s]->maxu2_bits = m;
}

void launch_group_max_u2(Scalars *const *scal, int n, cudaStream_t stream)
{
    GroupScal g;
    for (int s = 0; s < n && s < 64; ++s) g.p[s] = scal[s];
    group_max_u2_kernel<<<1, 1, 0, stream>>>(g, n);
}

// FP32C: the forward face state of direction d from the FP32 working array
// w into the face box c.fq (the reverse recomputes it instead of storing it).
void launch_face_state32(const Ctx &c, int d, const float *w)
{
    launch_face_eq_f2(face_eq_args<float, float>(c, d, w, make_phys<float>(c)), d, c.stream);
}

void launch_stage(const Ctx &c, int stage)
{
    if (c.prec == GKS_FP64 && c.fp64_ds && !c.gp_dir[0])
        stage == 1 ? stage_impl<double, dsf, 1>(c) : stage_impl<double, dsf, 2>(c);
    else if (c.prec == GKS_FP64)
        stage == 1 ? stage_impl<double, double, 1>(c) : stage_impl<double, double, 2>(c);
    else
        stage == 1 ? stage_impl<float, float, 1>(c) : stage_impl<float, float, 2>(c);
}

void launch_cfl(const Ctx &c)
{
    mark(c, K_MISC, 1);
    dt_kernel<<<1, 1, 0, c.stream>>>(c.scal, c.cfl, c.dt_fixed, c.hmin, c.csound);
    mark(c, K_MISC, 0);
}

void launch_advance(const Ctx &c)
{
    mark(c, K_MISC, 1);
    advance_kernel<<<1, 1, 0, c.stream>>>(c.scal);
    mark(c, K_MISC, 0);
}

void launch_scatter_state(const Ctx &c, const double *d_src)
{
    dim3 blk(32, 8), g((c.n[0] + 31) / 32, (c.n[1] + 7) / 8, (c.n[2] + kPrepZ - 1) / kPrepZ);
    scatter_kernel<<<g, blk, 0, c.stream>>>(c.prec, d_src, c.state, c.np, c.n[0], c.n[1], c.n[2], c.P[0], c.P[1],
                                            nullptr, 0.0f, nullptr);
}

void launch_scatter_state_prep(const Ctx &c, const double *d_src)
{
    cudaMemsetAsync(&c.scal->maxu2_bits, 0, sizeof(unsigned long long), c.stream);
    dim3 blk(32, 8), g((c.n[0] + 31) / 32, (c.n[1] + 7) / 8, (c.n[2] + kPrepZ - 1) / kPrepZ);
    scatter_kernel<<<g, blk, 0, c.stream>>>(c.prec, d_src, c.state, c.np, c.n[0], c.n[1], c.n[2], c.P[0], c.P[1],
                                            c.prec == GKS_FP32C ? (float *)c.wk0 : nullptr, (float)c.off, c.scal);
}

void launch_gather_state(const Ctx &c, double *d_dst)
{
    dim3 blk(32, 8), g((c.n[0] + 31) / 32, (c.n[1] + 7) / 8, c.n[2]);
    gather_kernel<<<g, blk, 0, c.stream>>>(c.prec, c.state, d_dst, c.np, c.n[0], c.n[1], c.n[2],
                                           c.P[0], c.P[1]);
}

void launch_fill_rest(const Ctx &c)
{
    dim3 blk(32, 8), g((c.n[0] + 31) / 32, (c.n[1] + 7) / 8, c.n[2]);
    fill_rest_kernel<<<g, blk, 0, c.stream>>>(c.prec, c.state, c.np, c.n[0], c.n[1], c.n[2], c.P[0],
                                              c.P[1]);
}

void launch_raw_copy(const Ctx &c, void *compact, int to_compact)
{
    dim3 blk(32, 8), g((c.n[0] + 31) / 32, (c.n[1] + 7) / 8, c.n[2]);
    if (c.prec == GKS_FP64)
        raw_copy_kernel<double><<<g, blk, 0, c.stream>>>((double *)c.state, (double *)compact, 4, c.np,
                                                         c.n[0], c.n[1], c.n[2], c.P[0], c.P[1],
                                                         to_compact);
    else
        raw_copy_kernel<float><<<g, blk, 0, c.stream>>>((float *)c.state, (float *)compact, 8, c.np,
                                                        c.n[0], c.n[1], c.n[2], c.P[0], c.P[1],
                                                        to_compact);
}

// FP32 values as FP64: out[i] = a[i] (+ b[i]) (+ off0 for i < n0), i < n.
__global__ void __launch_bounds__(256) widen_kernel(const float *a, const float *b, double *out, long n, long n0,
                                                     double off0)
{
    for (long i = blockIdx.x * 256L + threadIdx.x; i < n; i += (long)gridDim.x * 256L) {
        double v = (double)a[i];
        if (b) v += (double)b[i];
        if (i < n0) v += off0;
        out[i] = v;
    }
}

void launch_widen(const Ctx &c, const float *a, const float *b, double *out, long n, long n0, double off0)
{
    mark(c, K_MISC, 1);
    const long nb = (n + 255) / 256;
    widen_kernel<<<(int)(nb < 16L * sm_count() ? nb : 16L * sm_count()), 256, 0, c.stream>>>(a, b, out, n, n0, off0);
    mark(c, K_MISC, 0);
}

void launch_diagnostics(const Ctx &c, double *d_out5)
{
    const int nb = reduce_blocks(c.ncell);
    diag_partial_kernel<<<nb, 256, 0, c.stream>>>(c.prec, c.state, c.np, c.n[0], c.n[1], c.n[2],
                                                  c.P[0], c.P[1], c.h64[0], c.h64[1], c.h64[2],
                                                  c.partials);
    diag_final_kernel<<<1, 256, 0, c.stream>>>(c.partials, nb, d_out5);
}

int bounds_flag_stencil() { return bounds_flag_take(); }

}  // namespace gks
