// gks_adjoint.cu -- hand-written reverse mode (adjoint) of one S2O4 step
// (FP64 or FP32C), for gradients of a functional of the state with respect to the
// per-point actuator force scales and the inflow speed.
//
// The forward step (Sec. 2 and the end of Sec. 3.2) is a composition of
//   ghost fill G, spatial operator (L, Lt) = S(A) per direction d
//   [face state: WENO5 + half-space equilibrium + normal slope;
//    face flux: tangential quartic to the Gauss points + closed-form flux;
//    divergence], the two stage combinations, the ALM forcing
//   [trilinear sample, loads, truncated-Gaussian projection] and the IBM
//   direct forcing. The forward step (recorded, or recomputed from W^n)
//   keeps the Gauss-point inputs of every face of each stage and direction.
//   Its adjoint runs the pieces backwards. Every transposed stencil is
//   written as a gather (each
//   output sums its inputs in a fixed order), so the adjoint is
//   deterministic and uses no atomics on the state:
//   RA  per Gauss point of an interior face: reverse the flux (16 input
//       adjoints from the recorded inputs, which stay as they are);
//   RB  t2 transpose: Gauss adjoints -> adjoints of the t1-pass rows;
//   RC  t1 transpose: rows -> adjoints of Q0 and its normal slope per face;
//   RD  marching along d: paired WENO5 forward and reverse per cell, the
//       equilibrium and normal-slope reverse per face -> adjoints of the
//       6 cells of each face's stencil;
//   RE  per cell: gather the 6 faces whose stencil holds the cell;
//   ghost adjoint: axes z, y, x, one launch per side and layer, each ghost
//       adjoint added to its source cell (Riemann inflow through its
//       Jacobian; its U_inf sensitivity stored per ghost and reduced in a
//       fixed order).
// RA-RE run in a compute type T: double, or float (FP32 arithmetic and
// FP32 intermediate adjoints; the state adjoints and their sums in FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "gks_bounds.cuh"
#include "gks_device.cuh"
#include "gks_internal.h"

namespace gks {
namespace {

using namespace dev;

constexpr double kPi = 3.14159265358979323846;
constexpr double kS3 = 1.7320508075688772935;

// Explicit 5-point weights (offsets -2..2) of the tangential quartic at the
// Gauss points -g (index 0) and +g (index 1): values WV and derivatives WD.
__device__ __constant__ double cWV[2][5] = {
    {-1.0 / 4320.0 - 7.0 * kS3 / 432.0, 1.0 / 1080.0 + 25.0 * kS3 / 216.0, 719.0 / 720.0,
     1.0 / 1080.0 - 25.0 * kS3 / 216.0, -1.0 / 4320.0 + 7.0 * kS3 / 432.0},
    {-1.0 / 4320.0 + 7.0 * kS3 / 432.0, 1.0 / 1080.0 - 25.0 * kS3 / 216.0, 719.0 / 720.0,
     1.0 / 1080.0 + 25.0 * kS3 / 216.0, -1.0 / 4320.0 - 7.0 * kS3 / 432.0}};
__device__ __constant__ double cWD[2][5] = {
    {1.0 / 12.0 + kS3 / 54.0, -2.0 / 3.0 - 13.0 * kS3 / 54.0, 4.0 * kS3 / 9.0, 2.0 / 3.0 - 13.0 * kS3 / 54.0,
     -1.0 / 12.0 + kS3 / 54.0},
    {1.0 / 12.0 - kS3 / 54.0, -2.0 / 3.0 + 13.0 * kS3 / 54.0, -4.0 * kS3 / 9.0, 2.0 / 3.0 + 13.0 * kS3 / 54.0,
     -1.0 / 12.0 - kS3 / 54.0}};

// The same weights in FP32 for the FP32C reverse (no conversion at each use).
__device__ __constant__ float cWV32[2][5] = {
    {(float)(-1.0 / 4320.0 - 7.0 * kS3 / 432.0), (float)(1.0 / 1080.0 + 25.0 * kS3 / 216.0), (float)(719.0 / 720.0),
     (float)(1.0 / 1080.0 - 25.0 * kS3 / 216.0), (float)(-1.0 / 4320.0 + 7.0 * kS3 / 432.0)},
    {(float)(-1.0 / 4320.0 + 7.0 * kS3 / 432.0), (float)(1.0 / 1080.0 - 25.0 * kS3 / 216.0), (float)(719.0 / 720.0),
     (float)(1.0 / 1080.0 + 25.0 * kS3 / 216.0), (float)(-1.0 / 4320.0 - 7.0 * kS3 / 432.0)}};
__device__ __constant__ float cWD32[2][5] = {
    {(float)(1.0 / 12.0 + kS3 / 54.0), (float)(-2.0 / 3.0 - 13.0 * kS3 / 54.0), (float)(4.0 * kS3 / 9.0),
     (float)(2.0 / 3.0 - 13.0 * kS3 / 54.0), (float)(-1.0 / 12.0 + kS3 / 54.0)},
    {(float)(1.0 / 12.0 - kS3 / 54.0), (float)(-2.0 / 3.0 + 13.0 * kS3 / 54.0), (float)(-4.0 * kS3 / 9.0),
     (float)(2.0 / 3.0 + 13.0 * kS3 / 54.0), (float)(-1.0 / 12.0 - kS3 / 54.0)}};

__device__ __forceinline__ long lin(const int P0, const int P1, int i, int j, int k)
{
    return (long)(i + G) + (long)P0 * ((long)(j + G) + (long)P1 * (k + G));
}

// ------------------------------------------------------ reverse building blocks

// Adjoint of dev::gk_flux: given the adjoints of F0 (if needF0) and F1,
// accumulate the adjoints of its inputs (index-space tangential slopes).
template <typename T>
__device__ __forceinline__ void gk_flux_rev(const Phys<T> &ph, const T q[4], const T Dn[4], const T D1[4],
                                            const T D2[4], T ih1, T ih2, const T lF0[4], const T lF1[4],
                                            bool needF0, T qb[4], T Dnb[4], T D1b[4], T D2b[4])
{
    const T rho = ph.off + q[0];
    const T inv = T(1.0) / rho;
    const T invi[3] = {inv, inv * ih1, inv * ih2};
    const T *D[3] = {Dn, D1, D2};
    const T U[3] = {q[1] * inv, q[2] * inv, q[3] * inv};
    T g[3], Gm[3][3];
    for (int i = 0; i < 3; ++i) {
        g[i] = D[i][0] * invi[i];
        for (int j = 0; j < 3; ++j) Gm[i][j] = (D[i][j + 1] - U[j] * D[i][0]) * invi[i];
    }
    const T th = ph.theta, tl = T(2.0) * ph.lambda, mu = ph.mu;
    const T A0 = -(U[0] * g[0] + U[1] * g[1] + U[2] * g[2]) - (Gm[0][0] + Gm[1][1] + Gm[2][2]);
    T A[3];
    for (int k = 0; k < 3; ++k) A[k] = -g[k] - tl * (U[0] * Gm[0][k] + U[1] * Gm[1][k] + U[2] * Gm[2][k]);

    const T z0 = T(0.0);
    T rhob = z0, Ub[3] = {z0, z0, z0}, gb[3] = {z0, z0, z0}, Gb[3][3] = {{z0, z0, z0}, {z0, z0, z0}, {z0, z0, z0}};
    T A0b = z0, Ab[3] = {z0, z0, z0}, qd[4] = {z0, z0, z0, z0};
    // F1[0] = rho (A0 U0 + th A_0)
    {
        const T T0 = A0 * U[0] + th * A[0];
        rhob += lF1[0] * T0;
        const T T0b = lF1[0] * rho;
        A0b += T0b * U[0];
        Ub[0] += T0b * A0;
        Ab[0] += T0b * th;
    }
    // F1[1+k] = rho (A0 (U0 U_k + th d_k0) + th (A_k U0 + A_0 U_k))
    for (int k = 0; k < 3; ++k) {
        const T c = U[0] * U[k] + (k == 0 ? th : T(0.0));
        const T Tk = A0 * c + th * (A[k] * U[0] + A[0] * U[k]);
        rhob += lF1[1 + k] * Tk;
        const T Tb = lF1[1 + k] * rho;
        A0b += Tb * c;
        Ub[0] += Tb * A0 * U[k];
        Ub[k] += Tb * A0 * U[0];
        Ab[k] += Tb * th * U[0];
        Ub[0] += Tb * th * A[k];
        Ab[0] += Tb * th * U[k];
        Ub[k] += Tb * th * A[0];
    }
    if (needF0) {
        qd[1] += lF0[0];
        qd[1] += lF0[1] * U[0];
        Ub[0] += lF0[1] * q[1];
        qd[0] += lF0[1] * th;
        Gb[0][0] += -T(2.0) * mu * lF0[1];
        for (int k = 1; k < 3; ++k) {
            qd[1] += lF0[1 + k] * U[k];
            Ub[k] += lF0[1 + k] * q[1];
            Gb[0][k] -= mu * lF0[1 + k];
            Gb[k][0] -= mu * lF0[1 + k];
        }
    }
    // A_k = -g_k - tl sum_i U_i G_ik
    for (int k = 0; k < 3; ++k) {
        gb[k] -= Ab[k];
        for (int i = 0; i < 3; ++i) {
            Ub[i] -= tl * Ab[k] * Gm[i][k];
            Gb[i][k] -= tl * Ab[k] * U[i];
        }
    }
    // A0 = -sum U_i g_i - sum G_ii
    for (int i = 0; i < 3; ++i) {
        Ub[i] -= A0b * g[i];
        gb[i] -= A0b * U[i];
        Gb[i][i] -= A0b;
    }
    T Db[3][4] = {{z0, z0, z0, z0}, {z0, z0, z0, z0}, {z0, z0, z0, z0}};
    T invb[3] = {z0, z0, z0};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            Db[i][j + 1] += Gb[i][j] * invi[i];
            Ub[j] -= Gb[i][j] * D[i][0] * invi[i];
            Db[i][0] -= Gb[i][j] * U[j] * invi[i];
            invb[i] += Gb[i][j] * (D[i][j + 1] - U[j] * D[i][0]);
        }
        Db[i][0] += gb[i] * invi[i];
        invb[i] += gb[i] * D[i][0];
    }
    T inv_b = invb[0] + invb[1] * ih1 + invb[2] * ih2;
    for (int j = 0; j < 3; ++j) {
        qd[j + 1] += Ub[j] * inv;
        inv_b += Ub[j] * q[j + 1];
    }
    rhob += -inv_b * inv * inv;
    qd[0] += rhob;
    for (int v = 0; v < 4; ++v) {
        qb[v] = qd[v];
        Dnb[v] = Db[0][v];
        D1b[v] = Db[1][v];
        D2b[v] = Db[2][v];
    }
}

// Adjoint of dev::weno5_pair (both face values of the centre cell of
// q[0..4], weights folded as in the forward): seeds sR for the right-face
// value and sL for the left-face value; the cell adjoints are added to out.
template <typename T>
__device__ __forceinline__ void weno5_pair_rev(const T q[5], T sR, T sL, T out[5])
{
    const T c13 = T(13.0) / T(12.0);
    const T a = q[0], b = q[1], c = q[2], d = q[3], e = q[4];
    const T t0 = a - T(2.0) * b + c, u0 = a - T(4.0) * b + T(3.0) * c;
    const T t1 = b - T(2.0) * c + d, u1 = b - d;
    const T t2 = c - T(2.0) * d + e, u2 = T(3.0) * c - T(4.0) * d + e;
    const T s0 = T(1e-6) + (c13 * t0 * t0 + T(0.25) * u0 * u0);
    const T s1 = T(1e-6) + (c13 * t1 * t1 + T(0.25) * u1 * u1);
    const T s2 = T(1e-6) + (c13 * t2 * t2 + T(0.25) * u2 * u2);
    const T S0 = s0 * s0, S1 = s1 * s1, S2 = s2 * s2;
    const T w02 = T(6.0) * (S0 * S2), S01 = S0 * S1, S12 = S1 * S2;
    // right face: 6 p_k on (a,b,c), (b,c,d), (c,d,e), weights S12, w02, 3 S01
    const T P0 = T(2.0) * a - T(7.0) * b + T(11.0) * c, P1 = -b + T(5.0) * c + T(2.0) * d, P2 = T(2.0) * c + T(5.0) * d - e;
    const T wr2 = T(3.0) * S01;
    const T iDR = T(1.0) / (T(6.0) * (S12 + w02 + wr2));
    const T right = (S12 * P0 + w02 * P1 + wr2 * P2) * iDR;
    // left face: mirrored candidates, weights S01, w02, 3 S12
    const T Q0 = T(2.0) * e - T(7.0) * d + T(11.0) * c, Q1 = -d + T(5.0) * c + T(2.0) * b, Q2 = T(2.0) * c + T(5.0) * b - a;
    const T wl2 = T(3.0) * S12;
    const T iDL = T(1.0) / (T(6.0) * (S01 + w02 + wl2));
    const T left = (S01 * Q0 + w02 * Q1 + wl2 * Q2) * iDL;
    // value = N / D: Nb = s / D, Db = -Nb value
    const T NRb = sR * iDR, DRb6 = -T(6.0) * NRb * right;
    const T NLb = sL * iDL, DLb6 = -T(6.0) * NLb * left;
    const T P0b = NRb * S12, P1b = NRb * w02, P2b = NRb * wr2;
    const T Q0b = NLb * S01, Q1b = NLb * w02, Q2b = NLb * wl2;
    const T S12b = (NRb * P0 + DRb6) + T(3.0) * (NLb * Q2 + DLb6);
    const T w02b = (NRb * P1 + DRb6) + (NLb * Q1 + DLb6);
    const T S01b = T(3.0) * (NRb * P2 + DRb6) + (NLb * Q0 + DLb6);
    const T S0b = T(6.0) * S2 * w02b + S1 * S01b;
    const T S1b = S2 * S12b + S0 * S01b;
    const T S2b = S1 * S12b + T(6.0) * S0 * w02b;
    const T s0b = T(2.0) * s0 * S0b, s1b = T(2.0) * s1 * S1b, s2b = T(2.0) * s2 * S2b;
    const T t0b = s0b * (T(2.0) * c13) * t0, u0b = s0b * T(0.5) * u0;
    const T t1b = s1b * (T(2.0) * c13) * t1, u1b = s1b * T(0.5) * u1;
    const T t2b = s2b * (T(2.0) * c13) * t2, u2b = s2b * T(0.5) * u2;
    out[0] += t0b + u0b + T(2.0) * P0b - Q2b;
    out[1] += -T(2.0) * t0b - T(4.0) * u0b + t1b + u1b - T(7.0) * P0b - P1b + T(2.0) * Q1b + T(5.0) * Q2b;
    out[2] += t0b + T(3.0) * u0b - T(2.0) * t1b + t2b + T(3.0) * u2b + T(11.0) * P0b + T(5.0) * P1b + T(2.0) * P2b + T(11.0) * Q0b +
              T(5.0) * Q1b + T(2.0) * Q2b;
    out[3] += t1b - u1b - T(2.0) * t2b - T(4.0) * u2b + T(2.0) * P1b + T(5.0) * P2b - T(7.0) * Q0b - Q1b;
    out[4] += t2b + u2b - P2b + T(2.0) * Q0b;
}

// Adjoint of the half-space equilibrium state (local frame).
template <typename T>
__device__ __forceinline__ void equilibrium_rev(const Phys<T> &ph, const T Ql[4], const T Qr[4], const T Q0b[4],
                                                T Qlb[4], T Qrb[4])
{
    const T off = ph.off;
    const T rl = off + Ql[0], rr = off + Qr[0];
    const T irl = T(1.0) / rl, irr = T(1.0) / rr;
    const T Ul = Ql[1] * irl, Ur = Qr[1] * irr;
    // erf(z) and exp(-z^2) with z = sqrt(lambda) U, as in the forward
    T el, er, ml, mr, exl, exr;
    half_space_terms(ph.sqlam * Ul, el, ml, exl);
    half_space_terms(ph.sqlam * Ur, er, mr, exr);
    const T Pl = T(0.5) + T(0.5) * el, Pr = T(0.5) - T(0.5) * er;
    const T El = ph.kE * exl, Er = ph.kE * exr;
    T Plb = T(0.0), Prb = T(0.0);
    for (int v = 0; v < 4; ++v) {
        Plb += Q0b[v] * Ql[v];
        Prb += Q0b[v] * Qr[v];
        Qlb[v] = Q0b[v] * Pl;
        Qrb[v] = Q0b[v] * Pr;
    }
    T elb = T(0.5) * Q0b[0] * off + T(0.5) * Plb;
    T erb = -T(0.5) * Q0b[0] * off - T(0.5) * Prb;
    Qlb[0] += Q0b[1] * El;
    Qrb[0] -= Q0b[1] * Er;
    const T Elb = Q0b[1] * Ql[0], Erb = -Q0b[1] * Qr[0];
    T xlb = Q0b[1] * off * ph.kE * exl + Elb * El;
    T xrb = -Q0b[1] * off * ph.kE * exr + Erb * Er;
    // d erf(z)/dz = (2/sqrt pi) exp(-z^2), and z^2 = lambda U^2: exp(-z^2) = exp(x)
    const T dz = T(2.0) / T(T(1.7724538509055160273));
    T Ulb = elb * ph.sqlam * dz * exl + xlb * (-T(2.0) * ph.lambda * Ul);
    T Urb = erb * ph.sqlam * dz * exr + xrb * (-T(2.0) * ph.lambda * Ur);
    Qlb[1] += Ulb * irl;
    Qlb[0] += -Ulb * Ul * irl;
    Qrb[1] += Urb * irr;
    Qrb[0] += -Urb * Ur * irr;
}

// The constants of ph in the compute type T of a reverse kernel.
template <typename T>
__device__ __forceinline__ Phys<T> phys_as(const Phys<double> &p)
{
    Phys<T> q;
    q.lambda = T(p.lambda);
    q.theta = T(p.theta);
    q.mu = T(p.mu);
    q.off = T(p.off);
    q.sqlam = T(p.sqlam);
    q.kE = T(p.kE);
    return q;
}

// WENO5 pair of a 5-cell stencil in compute type T on the cells minus the
// centre cell (both face values shift with it and the reverse depends on
// differences only), so that FP32 keeps the relative precision of the
// differences of FP64 states.
template <typename T>
__device__ __forceinline__ void pair_values(const double q[5], double &right, double &left)
{
    T qs[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) qs[k] = T(q[k] - q[2]);
    T r, l;
    weno5_pair(qs, r, l);
    right = q[2] + (double)r;
    left = q[2] + (double)l;
}

template <typename T>
__device__ __forceinline__ void pair_rev(const double q[5], double sR, double sL, double out[5])
{
    T qs[5], o[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k < 5; ++k) qs[k] = T(q[k] - q[2]);
    weno5_pair_rev<T>(qs, T(sR), T(sL), o);
#pragma unroll
    for (int k = 0; k < 5; ++k) out[k] += (double)o[k];
}

// equilibrium_rev in compute type T with FP64 arguments.
template <typename T>
__device__ __forceinline__ void equilibrium_rev_as(const Phys<double> &ph, const double Ql[4], const double Qr[4],
                                                   const double Q0b[4], double Qlb[4], double Qrb[4])
{
    const Phys<T> pt = phys_as<T>(ph);
    T l[4], r[4], b[4], lb[4], rb[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        l[v] = T(Ql[v]);
        r[v] = T(Qr[v]);
        b[v] = T(Q0b[v]);
    }
    equilibrium_rev<T>(pt, l, r, b, lb, rb);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        Qlb[v] = (double)lb[v];
        Qrb[v] = (double)rb[v];
    }
}

// ------------------------------------------------------------------ kernels

struct RevArgs {
    const double *A;          // forward working array (ghost-filled, padded)
    const float *Ahi, *Alo;   // FP32 reverse: A as hi + lo floats
    long nfq;                 // component stride of the face-box adjoints
    int e1p;
    const double *lamL, *lamLt;   // padded indexing; lamL may be null (stage 2)
    // the recorded Gauss-point inputs (read only) and the adjoints inside the
    // spatial adjoint of one direction, in the reverse's compute type:
    // Gauss-point inputs, t1-pass rows, face boxes, per-face cell slots
    void *lamG;
    void *lamGa;
    long nG;
    void *lamR;
    long nR;
    void *lamFQ, *lamC;
    double *lamA;
    const double *ihd, *ih1, *ih2, *ihf;
    int n[3], P[3];
    int d, t1, t2, nd, n1, n2;
    long np;
    Phys<double> ph;
};

// RA: reverse of the face flux at every interior face: from the 16 recorded
// inputs of each Gauss point (lamG, only read) their adjoints (lamGa, same
// layout). A thread takes one Gauss point g of one face (block: 32 faces
// along t1 x 2 along t2 x the 4 Gauss points), so that a face's 4 points run
// side by side and share the cell-adjoint loads through L1.
constexpr int kRevFluxB = 2;   // faces along t2 per block

template <typename T>
__global__ void __launch_bounds__(256) rev_flux_kernel(RevArgs A)
{
    const int g = threadIdx.y & 3;
    const int a = blockIdx.x * 32 + threadIdx.x, b = blockIdx.y * kRevFluxB + (threadIdx.y >> 2), f = blockIdx.z;
    if (a >= A.n1 || b >= A.n2) return;
    // adjoint of the face-averaged fluxes from the two neighbour cells
    const int gc[4] = {0, 1 + A.d, 1 + A.t1, 1 + A.t2};
    T sF0[4] = {0, 0, 0, 0}, sF1[4] = {0, 0, 0, 0};
    int cl[3], cr[3];
    cl[A.d] = f - 1; cl[A.t1] = a; cl[A.t2] = b;
    cr[A.d] = f; cr[A.t1] = a; cr[A.t2] = b;
    const bool hasl = f - 1 >= 0, hasr = f < A.nd;
    const long il = lin(A.P[0], A.P[1], cl[0], cl[1], cl[2]), ir = lin(A.P[0], A.P[1], cr[0], cr[1], cr[2]);
    if (!in_bounds(il, A.np) || !in_bounds(ir, A.np) || !in_bounds(((long)f * A.n2 + b) * A.n1 + a, A.nG)) return;
    const T ihl = hasl ? T(A.ihd[f - 1 + G]) : T(0), ihr = hasr ? T(A.ihd[f + G]) : T(0);
    for (int v = 0; v < 4; ++v) {
        const long o = gc[v] * A.np;
        const T ll = hasl ? T(A.lamLt[o + il]) : T(0), lr = hasr ? T(A.lamLt[o + ir]) : T(0);
        sF1[v] = T(0.25) * (-ll * ihl + lr * ihr);
        if (A.lamL) {
            const T ml = hasl ? T(A.lamL[o + il]) : T(0), mr = hasr ? T(A.lamL[o + ir]) : T(0);
            sF0[v] = T(0.25) * (-ml * ihl + mr * ihr);
        }
    }
    const T ih1 = T(A.ih1[a + G]), ih2 = T(A.ih2[b + G]);
    const Phys<T> ph = phys_as<T>(A.ph);
    const long face = ((long)f * A.n2 + b) * A.n1 + a;
    const T *in = (const T *)A.lamG + (long)(16 * g) * A.nG + face;
    T *io = (T *)A.lamGa + (long)(16 * g) * A.nG + face;
    T q[4], Dn[4], D1[4], D2[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        q[v] = in[v * A.nG];
        Dn[v] = in[(4 + v) * A.nG];
        D1[v] = in[(8 + v) * A.nG];
        D2[v] = in[(12 + v) * A.nG];
    }
    T qb[4], Dnb[4], D1b[4], D2b[4];
    gk_flux_rev<T>(ph, q, Dn, D1, D2, ih1, ih2, sF0, sF1, A.lamL != nullptr, qb, Dnb, D1b, D2b);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        io[v * A.nG] = qb[v];
        io[(4 + v) * A.nG] = Dnb[v];
        io[(8 + v) * A.nG] = D1b[v];
        io[(12 + v) * A.nG] = D2b[v];
    }
}

// RB: transpose of the t2 pass: for every t1-pass row (f, a, b'), b' in
// [-2, n2+2), t1 Gauss point m and component v, the 5-tap gathers over the
// faces b = b'-2 .. b'+2 of the Gauss-point adjoints (value and t2 slope into
// the Q0 row, t1 slope into the t1-derivative row, normal slope into the slope
// row). A thread owns (a, m, v) of one face plane and walks kRevT2 rows of b'
// with the 8 adjoints of the 5 faces in a register window, so that every face
// value is read once.
constexpr int kRevT2 = 32;

template <typename T>
__global__ void __launch_bounds__(256) rev_t2_kernel(RevArgs A)
{
    const int a = blockIdx.x * 32 + threadIdx.x;
    const int mv = threadIdx.y, m = mv >> 2, v = mv & 3;   // 8 = 2 Gauss points x 4 components
    const int f = blockIdx.z, bp0 = (int)blockIdx.y * kRevT2 - 2;
    if (a >= A.n1) return;
    const int bp1 = min(bp0 + kRevT2, A.n2 + 2);
    const long nG = A.nG;
    // per face b: Q0 adjoints of the two t2 points (0, 1), t2 slopes (2, 3),
    // t1 slopes (4, 5), normal slopes (6, 7) of Gauss points g = 2m + nn
    auto load = [&](int b, T x[8]) {
        if (b < 0 || b >= A.n2) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = T(0);
            return;
        }
        if (!in_bounds(((long)f * A.n2 + b) * A.n1 + a, nG)) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = T(0);
            return;
        }
        const T *Gf = (const T *)A.lamGa + ((long)f * A.n2 + b) * A.n1 + a;
#pragma unroll
        for (int nn = 0; nn < 2; ++nn) {
            const long g16 = 16L * (2 * m + nn);
            x[nn] = T(Gf[(g16 + 0 + v) * nG]);
            x[2 + nn] = T(Gf[(g16 + 12 + v) * nG]);
            x[4 + nn] = T(Gf[(g16 + 8 + v) * nG]);
            x[6 + nn] = T(Gf[(g16 + 4 + v) * nG]);
        }
    };
    T win[5][8];   // faces b' - 2 .. b' + 2
#pragma unroll
    for (int k = 0; k < 4; ++k) load(bp0 - 2 + k, win[k + 1]);
    for (int bp = bp0; bp < bp1; ++bp) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int e = 0; e < 8; ++e) win[k][e] = win[k + 1][e];
        load(bp + 2, win[4]);
        T X = T(0), Y = T(0), Z = T(0);
#pragma unroll
        for (int k = 0; k < 5; ++k) {   // face b = bp - 2 + k, stencil offset s = bp - b + 2 = 4 - k
#pragma unroll
            for (int nn = 0; nn < 2; ++nn) {
                const T wv = T(cWV[nn][4 - k]), wd = T(cWD[nn][4 - k]);
                X += wv * win[k][nn] + wd * win[k][2 + nn];
                Y += wv * win[k][4 + nn];
                Z += wv * win[k][6 + nn];
            }
        }
        const long row = ((long)f * (A.n2 + 4) + (bp + 2)) * A.n1 + a;
        if (!in_bounds(row, A.nR)) continue;
        T *lr = (T *)A.lamR;
        lr[(0 * 8 + m * 4 + v) * A.nR + row] = X;
        lr[(1 * 8 + m * 4 + v) * A.nR + row] = Y;
        lr[(2 * 8 + m * 4 + v) * A.nR + row] = Z;
    }
}

// RC: transpose of the t1 pass, per face of the extended box.
template <typename T>
__global__ void __launch_bounds__(256) rev_t1_kernel(RevArgs A)
{
    const int ap = (int)(blockIdx.x * 32 + threadIdx.x) - 2, bp = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int f = blockIdx.z;
    if (ap >= A.n1 + 2 || bp >= A.n2 + 2) return;
    T lq[4] = {0, 0, 0, 0}, ln[4] = {0, 0, 0, 0};
    const T *lr = (const T *)A.lamR;
    const int alo = ap - 2 < 0 ? 0 : ap - 2, ahi = ap + 2 > A.n1 - 1 ? A.n1 - 1 : ap + 2;
    for (int a = alo; a <= ahi; ++a) {
        const int r = ap - a + 2;
        const long row = ((long)f * (A.n2 + 4) + (bp + 2)) * A.n1 + a;
        if (!in_bounds(row, A.nR)) continue;
        for (int m = 0; m < 2; ++m) {
            const T wv = T(cWV[m][r]), wd = T(cWD[m][r]);
            for (int v = 0; v < 4; ++v) {
                lq[v] += wv * lr[(0 * 8 + m * 4 + v) * A.nR + row] + wd * lr[(1 * 8 + m * 4 + v) * A.nR + row];
                ln[v] += wv * lr[(2 * 8 + m * 4 + v) * A.nR + row];
            }
        }
    }
    const long o = ((long)f * (A.n2 + 4) + (bp + 2)) * A.e1p + (ap + 2);
    if (!in_bounds(o, A.nfq)) return;
    T *fq = (T *)A.lamFQ;
    for (int v = 0; v < 4; ++v) {
        fq[v * A.nfq + o] = lq[v];
        fq[(4 + v) * A.nfq + o] = ln[v];
    }
}

// RD: reverse of WENO5, the equilibrium state and the normal slope. Each
// thread walks kRevMarch faces along d at one position of the extended
// tangential box with the 6 cells f-3 .. f+2 in registers. Face f's slots
// of lamC (cells f-3 .. f+2) take its normal-slope adjoint and the paired
// WENO5 reverse of cell f-1 (seeds: its left value from face f-1, its right
// value from face f); the last face also takes cell f's reverse (left value
// only). The sum over faces per cell (RE) is the same as with one reverse
// per face side.
constexpr int kRevMarch = 16;

__global__ void __launch_bounds__(256) rev_face_state_kernel(RevArgs A)
{
    using T = double;
    const double *lamFQ = (const double *)A.lamFQ;
    double *lamC = (double *)A.lamC;
    const int a = (int)(blockIdx.x * 32 + threadIdx.x) - 2, b = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int nf = A.nd + 1, f0 = blockIdx.z * kRevMarch;
    if (a >= A.n1 + 2 || b >= A.n2 + 2 || f0 >= nf) return;
    const int f1 = min(f0 + kRevMarch, nf);
    const long stride[3] = {1, (long)A.P[0], (long)A.P[0] * A.P[1]};
    const long sd = stride[A.d];
    int cc[3];
    cc[A.d] = 0; cc[A.t1] = a; cc[A.t2] = b;
    const long base = lin(A.P[0], A.P[1], cc[0], cc[1], cc[2]);   // cell 0 along d
    // cells f0-4 .. f1+1 are read, faces f0-1 .. f1-1 read and written
    if (!in_bounds(base + (long)(f0 - 4 < -G ? -G : f0 - 4) * sd, A.np) || !in_bounds(base + (long)(f1 + 1) * sd, A.np) ||
        !in_bounds(((long)(f0 > 0 ? f0 - 1 : 0) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq) ||
        !in_bounds(((long)(f1 - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq))
        return;
    const int comp[4] = {0, 1 + A.d, 1 + A.t1, 1 + A.t2};
    // window w[v][k] = cell f-3+k at face f; before the first face: cells f0-4 .. f0+1
    double w[4][6];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int cell = f0 - 4 + k;
            w[v][k] = cell >= -G ? A.A[comp[v] * A.np + base + (long)cell * sd] : 0.0;
        }
    // carried: right value of cell f-1 and the left-value seed of cell f-1
    double Rprev[4], Sprev[4];
    {
        double lft[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) pair_values<T>(&w[v][1], Rprev[v], lft[v]);   // cell f0-1
        if (f0 == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v) Sprev[v] = 0.0;
        } else {
            double Rpp[4], dum;
#pragma unroll
            for (int v = 0; v < 4; ++v) pair_values<T>(&w[v][0], Rpp[v], dum);    // cell f0-2
            const long o = ((long)(f0 - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
            double Q0b[4], Qlb[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) Q0b[v] = lamFQ[v * A.nfq + o];
            equilibrium_rev_as<T>(A.ph, Rpp, lft, Q0b, Qlb, Sprev);
        }
    }
    for (int f = f0; f < f1; ++f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
#pragma unroll
            for (int k = 0; k < 5; ++k) w[v][k] = w[v][k + 1];
            w[v][5] = A.A[comp[v] * A.np + base + (long)(f + 2) * sd];
        }
        double Ql[4], Qr[4], Rt[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Ql[v] = Rprev[v];
            pair_values<T>(&w[v][1], Rt[v], Qr[v]);   // cell f
        }
        const long o = ((long)f * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
        double Q0b[4], DNb[4], Qlb[4], Qrb[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Q0b[v] = lamFQ[v * A.nfq + o];
            DNb[v] = lamFQ[(4 + v) * A.nfq + o];
        }
        equilibrium_rev_as<T>(A.ph, Ql, Qr, Q0b, Qlb, Qrb);
        const double s = A.ihf[f] * (1.0 / 12.0);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double cb[6] = {0, 0, 0, 0, 0, 0};
            cb[1] += DNb[v] * s;
            cb[2] -= 15.0 * DNb[v] * s;
            cb[3] += 15.0 * DNb[v] * s;
            cb[4] -= DNb[v] * s;
            pair_rev<T>(&w[v][0], Qlb[v], Sprev[v], &cb[0]);      // cell f-1
            if (f == nf - 1) pair_rev<T>(&w[v][1], 0.0, Qrb[v], &cb[1]);   // cell f, left value only
#pragma unroll
            for (int m = 0; m < 6; ++m) lamC[(m * 4 + v) * A.nfq + o] = cb[m];
            Rprev[v] = Rt[v];
            Sprev[v] = Qrb[v];
        }
    }
}

// The WENO5 pair in FP32 of 5 cells given as hi + lo floats, on the cells
// minus the centre cell: (hi_k - hi_2) + (lo_k - lo_2) keeps the precision of
// the FP64 differences (the hi difference of nearby values is exact).
__device__ __forceinline__ void diffs32(const float hi[5], const float lo[5], float qs[5])
{
#pragma unroll
    for (int k = 0; k < 5; ++k) qs[k] = (hi[k] - hi[2]) + (lo[k] - lo[2]);
}

__device__ __forceinline__ void pair_values32(const float hi[5], const float lo[5], float &right, float &left)
{
    float qs[5], r, l;
    diffs32(hi, lo, qs);
    weno5_pair(qs, r, l);
    right = hi[2] + (lo[2] + r);
    left = hi[2] + (lo[2] + l);
}

__device__ __forceinline__ void pair_rev32(const float hi[5], const float lo[5], float sR, float sL, float out[5])
{
    float qs[5];
    diffs32(hi, lo, qs);
    weno5_pair_rev<float>(qs, sR, sL, out);
}

// RD in FP32 (the FP32 reverse): the same march as rev_face_state_kernel on
// the working array split into hi + lo floats, with FP32 face-box adjoints in
// and FP32 cell slots out.
template <bool LO>
__global__ void __launch_bounds__(256) rev_face_state32_kernel(RevArgs A)
{
    const float *lamFQ = (const float *)A.lamFQ;
    float *lamC = (float *)A.lamC;
    const int a = (int)(blockIdx.x * 32 + threadIdx.x) - 2, b = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int nf = A.nd + 1, f0 = blockIdx.z * kRevMarch;
    if (a >= A.n1 + 2 || b >= A.n2 + 2 || f0 >= nf) return;
    const int f1 = min(f0 + kRevMarch, nf);
    const long stride[3] = {1, (long)A.P[0], (long)A.P[0] * A.P[1]};
    const long sd = stride[A.d];
    int cc[3];
    cc[A.d] = 0; cc[A.t1] = a; cc[A.t2] = b;
    const long base = lin(A.P[0], A.P[1], cc[0], cc[1], cc[2]);
    // cells f0-4 .. f1+1 are read, faces f0-1 .. f1-1 read and written
    if (!in_bounds(base + (long)(f0 - 4 < -G ? -G : f0 - 4) * sd, A.np) || !in_bounds(base + (long)(f1 + 1) * sd, A.np) ||
        !in_bounds(((long)(f0 > 0 ? f0 - 1 : 0) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq) ||
        !in_bounds(((long)(f1 - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq))
        return;
    const int comp[4] = {0, 1 + A.d, 1 + A.t1, 1 + A.t2};
    const Phys<float> ph = phys_as<float>(A.ph);
    float wh[4][6], wl[4][6];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int cell = f0 - 4 + k;
            const long l = comp[v] * A.np + base + (long)cell * sd;
            wh[v][k] = cell >= -G ? A.Ahi[l] : 0.0f;
            wl[v][k] = (LO && cell >= -G) ? A.Alo[l] : 0.0f;
        }
    float Rprev[4], Sprev[4];
    {
        float lft[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) pair_values32(&wh[v][1], &wl[v][1], Rprev[v], lft[v]);   // cell f0-1
        if (f0 == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v) Sprev[v] = 0.0f;
        } else {
            float Rpp[4], dum;
#pragma unroll
            for (int v = 0; v < 4; ++v) pair_values32(&wh[v][0], &wl[v][0], Rpp[v], dum);    // cell f0-2
            const long o = ((long)(f0 - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
            float Q0b[4], Qlb[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) Q0b[v] = lamFQ[v * A.nfq + o];
            equilibrium_rev<float>(ph, Rpp, lft, Q0b, Qlb, Sprev);
        }
    }
    for (int f = f0; f < f1; ++f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                wh[v][k] = wh[v][k + 1];
                wl[v][k] = wl[v][k + 1];
            }
            const long l = comp[v] * A.np + base + (long)(f + 2) * sd;
            wh[v][5] = A.Ahi[l];
            wl[v][5] = LO ? A.Alo[l] : 0.0f;
        }
        float Ql[4], Qr[4], Rt[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Ql[v] = Rprev[v];
            pair_values32(&wh[v][1], &wl[v][1], Rt[v], Qr[v]);   // cell f
        }
        const long o = ((long)f * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
        float Q0b[4], DNb[4], Qlb[4], Qrb[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Q0b[v] = lamFQ[v * A.nfq + o];
            DNb[v] = lamFQ[(4 + v) * A.nfq + o];
        }
        equilibrium_rev<float>(ph, Ql, Qr, Q0b, Qlb, Qrb);
        const float s = (float)(A.ihf[f] * (1.0 / 12.0));
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float cb[6] = {0, 0, 0, 0, 0, 0};
            const float ds = DNb[v] * s;
            cb[1] += ds;
            cb[2] -= 15.0f * ds;
            cb[3] += 15.0f * ds;
            cb[4] -= ds;
            pair_rev32(&wh[v][0], &wl[v][0], Qlb[v], Sprev[v], &cb[0]);      // cell f-1
            if (f == nf - 1) pair_rev32(&wh[v][1], &wl[v][1], 0.0f, Qrb[v], &cb[1]);   // cell f, left value only
#pragma unroll
            for (int m = 0; m < 6; ++m) lamC[(m * 4 + v) * A.nfq + o] = cb[m];
            Rprev[v] = Rt[v];
            Sprev[v] = Qrb[v];
        }
    }
}

// RD and RE of an FP32C grid in one march: a thread owns the cells
// [c0, c0 + kRevCells) of one line along d (ghost cells included) and walks
// the faces c0 - 2 .. c0 + kRevCells + 2 that read them, with the 6 cells of
// the current face's stencil in registers (FP32 cells as the forward read
// them, density as rho - off) and their adjoints in a rolling window; a cell
// leaves the window after its last face (f = c + 3) and its adjoint, summed
// over its faces in face order as RE sums them, is added to lamA. Each cell
// is written by one thread. The face reverse is rev_face_state32_kernel's.
constexpr int kRevCells = 24;

__global__ void __launch_bounds__(256, 2) rev_face_cells32_kernel(RevArgs A)
{
    const float *lamFQ = (const float *)A.lamFQ;
    const int a = (int)(blockIdx.x * 32 + threadIdx.x) - 2, b = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int nf = A.nd + 1;
    const int c0 = (int)blockIdx.z * kRevCells - G, c1 = min(c0 + kRevCells, A.nd + G);
    if (a >= A.n1 + 2 || b >= A.n2 + 2 || c0 >= A.nd + G) return;
    const int fs = max(0, c0 - 2), fe = min(nf - 1, c1 + 2);   // faces [fs, fe]
    if (fs > fe) return;
    // padded strides by axis (selects, not an indexed local array)
    auto str = [&](int ax) -> long { return ax == 0 ? 1L : (ax == 1 ? (long)A.P[0] : (long)A.P[0] * A.P[1]); };
    const long sd = str(A.d);
    const long base = G * (1L + A.P[0] + (long)A.P[0] * A.P[1]) + (long)a * str(A.t1) + (long)b * str(A.t2);
    // cells fs-4 .. fe+2 are read, faces fs-1 .. fe read
    if (!in_bounds(base + (long)(fs - 4 < -G ? -G : fs - 4) * sd, A.np) || !in_bounds(base + (long)(fe + 2) * sd, A.np) ||
        !in_bounds(((long)(fs > 0 ? fs - 1 : 0) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq) ||
        !in_bounds(((long)fe * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2), A.nfq))
        return;
    const int comp[4] = {0, 1 + A.d, 1 + A.t1, 1 + A.t2};
    const Phys<float> ph = phys_as<float>(A.ph);
    const float zl[5] = {0, 0, 0, 0, 0};
    float wh[4][6];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int cell = fs - 4 + k;
            wh[v][k] = cell >= -G ? A.Ahi[comp[v] * A.np + base + (long)cell * sd] : 0.0f;
        }
    float Rprev[4], Sprev[4];
    {
        float lft[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) pair_values32(&wh[v][1], zl, Rprev[v], lft[v]);   // cell fs-1
        if (fs == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v) Sprev[v] = 0.0f;
        } else {
            float Rpp[4], dum;
#pragma unroll
            for (int v = 0; v < 4; ++v) pair_values32(&wh[v][0], zl, Rpp[v], dum);    // cell fs-2
            const long o = ((long)(fs - 1) * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
            float Q0b[4], Qlb[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) Q0b[v] = lamFQ[v * A.nfq + o];
            equilibrium_rev<float>(ph, Rpp, lft, Q0b, Qlb, Sprev);
        }
    }
    float acc[4][6];   // adjoints of the cells f-3 .. f+2 of the current face f
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[v][k] = 0.0f;
    // the cell entering the window, loaded one face ahead
    float nxt[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) nxt[v] = A.Ahi[comp[v] * A.np + base + (long)(fs + 2) * sd];
#pragma unroll 1
    for (int f = fs; f <= fe; ++f) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
#pragma unroll
            for (int k = 0; k < 5; ++k) wh[v][k] = wh[v][k + 1];
            wh[v][5] = nxt[v];
        }
        if (f < fe) {   // cell f + 3 <= fe + 2: inside the checked range
#pragma unroll
            for (int v = 0; v < 4; ++v) nxt[v] = A.Ahi[comp[v] * A.np + base + (long)(f + 3) * sd];
        }
        float Ql[4], Qr[4], Rt[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Ql[v] = Rprev[v];
            pair_values32(&wh[v][1], zl, Rt[v], Qr[v]);   // cell f
        }
        const long o = ((long)f * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
        float Q0b[4], DNb[4], Qlb[4], Qrb[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Q0b[v] = lamFQ[v * A.nfq + o];
            DNb[v] = lamFQ[(4 + v) * A.nfq + o];
        }
        equilibrium_rev<float>(ph, Ql, Qr, Q0b, Qlb, Qrb);
        const float s = (float)(A.ihf[f] * (1.0 / 12.0));
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float cb[6] = {0, 0, 0, 0, 0, 0};
            const float ds = DNb[v] * s;
            cb[1] += ds;
            cb[2] -= 15.0f * ds;
            cb[3] += 15.0f * ds;
            cb[4] -= ds;
            pair_rev32(&wh[v][0], zl, Qlb[v], Sprev[v], &cb[0]);      // cell f-1
            if (f == nf - 1) pair_rev32(&wh[v][1], zl, 0.0f, Qrb[v], &cb[1]);   // cell f, left value only
#pragma unroll
            for (int m = 0; m < 6; ++m) acc[v][m] += cb[m];
            Rprev[v] = Rt[v];
            Sprev[v] = Qrb[v];
        }
        // cell f-3 has had its last face: add it if this thread owns it
        const int cl = f - 3;
        if (cl >= c0 && cl < c1) {
#pragma unroll
            for (int v = 0; v < 4; ++v) A.lamA[comp[v] * A.np + base + (long)cl * sd] += (double)acc[v][0];
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[v][k] = acc[v][k + 1];
            acc[v][5] = 0.0f;
        }
    }
    // cells fe-2 .. fe+2 are still in the window (their faces beyond fe do not exist)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int cl = fe - 2 + k;
        if (cl >= c0 && cl < c1) {
#pragma unroll
            for (int v = 0; v < 4; ++v) A.lamA[comp[v] * A.np + base + (long)cl * sd] += (double)acc[v][k];
        }
    }
}

// A (FP64) as hi + lo floats for the FP32 face-state reverse.
__global__ void __launch_bounds__(256) split_kernel(const double *A, float *hi, float *lo, long n)
{
    for (long i = blockIdx.x * 256L + threadIdx.x; i < n; i += (long)gridDim.x * 256L) {
        const double x = A[i];
        const float h = (float)x;
        hi[i] = h;
        lo[i] = (float)(x - (double)h);
    }
}

// RE: gather, per cell of the padded box along d and the extended
// tangential box, the contributions of the 6 faces whose stencil holds it.
template <typename T>
__global__ void __launch_bounds__(256) rev_gather_cells_kernel(RevArgs A)
{
    const T *lamC = (const T *)A.lamC;
    const int a = (int)(blockIdx.x * 32 + threadIdx.x) - 2, b = (int)(blockIdx.y * 8 + threadIdx.y) - 2;
    const int c = (int)blockIdx.z - G;
    if (a >= A.n1 + 2 || b >= A.n2 + 2) return;
    const int comp[4] = {0, 1 + A.d, 1 + A.t1, 1 + A.t2};
    T acc[4] = {0, 0, 0, 0};
    const int flo = c - 2 < 0 ? 0 : c - 2, fhi = c + 3 > A.nd ? A.nd : c + 3;
    for (int f = flo; f <= fhi; ++f) {
        const int m = c - f + 3;
        const long o = ((long)f * (A.n2 + 4) + (b + 2)) * A.e1p + (a + 2);
        if (!in_bounds(o, A.nfq)) continue;
        for (int v = 0; v < 4; ++v) acc[v] += lamC[(m * 4 + v) * A.nfq + o];
    }
    int cc[3];
    cc[A.d] = c; cc[A.t1] = a; cc[A.t2] = b;
    const long l = lin(A.P[0], A.P[1], cc[0], cc[1], cc[2]);
    if (!in_bounds(l, A.np)) return;
    for (int v = 0; v < 4; ++v) A.lamA[comp[v] * A.np + l] += (double)acc[v];
}

// ------------------------------------------------ fused FP32C reverse (RA-RC)

// FP32C grids: RA, RB and RC of one direction in one pass over the 32 x 8
// face tiles of the forward, with the Gauss-point inputs and adjoints kept in
// shared memory. Per tile: the face box of the forward (recomputed from the
// recorded FP32 working array by the forward's face-state kernel) arrives by
// TMA and the forward's t1 pass fills the rows; each thread then takes one
// face, redoes its t2 pass and reverses the flux at its 4 Gauss points (the
// 64 input adjoints go to shared memory, over the dead face-box buffer);
// the transposed t2 pass (each row adjoint gathers the faces that read the
// row) and the transposed t1 pass (each face-box adjoint gathers the row
// columns that read it) give the adjoints of the tile's face box with its
// tangential halo, written as the tile's partial. Halos overlap the
// neighbouring tiles: sum_partials32_kernel adds the partials of a face in a
// fixed order.
struct Rev32Args {
    const double *lamL, *lamLt;       // padded cell adjoints; lamL null in stage 2
    const float *ihd, *ih1, *ih2;     // inverse cell widths along d, t1, t2 (padded index)
    float *part;                      // per tile: 8 x SQ_H x SQ_W face-box adjoints
    int n1, n2, nf, nd, d, t1, t2;
    long np, sd, s1, s2, base;        // padded strides along d, t1, t2; index of cell (0, 0, 0)
    Phys<float> ph;
    Scalars *scal;
};

constexpr int kPartN = 8 * SQ_H * SQ_W;   // face-box adjoints of one tile
constexpr int kGA = 64 * TX * TY;         // Gauss-point input adjoints of one tile

constexpr size_t rev_tile32_smem_bytes() { return (size_t)(kGA + ST_N) * sizeof(float) + 2 * sizeof(uint64_t); }
static_assert(SQ_N <= kGA, "the face-box tile lives in the Gauss-point adjoint buffer");

__global__ void __launch_bounds__(256, 2) rev_tile32_kernel(const __grid_constant__ CUtensorMap tmap, Rev32Args A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ga = reinterpret_cast<float *>(smem_raw);   // [64][TY][TX]
    float *sq = ga;                                     // face-box tile, dead after the t1 pass
    float *st = ga + kGA;                               // t1-pass rows, then their adjoints
    uint64_t *bar = reinterpret_cast<uint64_t *>(st + ST_N);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int NA = (A.n1 + TX - 1) / TX, NB = (A.n2 + TY - 1) / TY;
    const int ntiles = NA * NB * A.nf;
    const uint32_t bytes = (uint32_t)(SQ_N * sizeof(float));
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int gc[4] = {0, 1 + A.d, 1 + A.t1, 1 + A.t2};
    const bool needF0 = A.lamL != nullptr;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int ta = t % NA, tb = (t / NA) % NB, f = t / (NA * NB);
        if (tid == 0) {
            fence_proxy_async();
            tma_load_tile(&tmap, sq, &bar[0], ta * TX, tb * TY, f, bytes);
        }
        const bool ok = mbar_wait(&bar[0], (uint32_t)(k & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(&A.scal->flags, FLAG_TIMEOUT);
            return;
        }
        tile_t1_pass(sq, st, tid);
        __syncthreads();

        // RA: per face, the 4 Gauss points
        const int a = ta * TX + tx, b = tb * TY + ty;
        if (a < A.n1 && b < A.n2) {
            const bool hasl = f >= 1, hasr = f < A.nd;
            const long ir = A.base + (long)f * A.sd + (long)a * A.s1 + (long)b * A.s2, il = ir - A.sd;
            const bool okc = in_bounds(il, A.np) && in_bounds(ir, A.np);
            const float ihl = hasl ? A.ihd[f - 1 + G] : 0.0f, ihr = hasr ? A.ihd[f + G] : 0.0f;
            float sF0[4] = {0, 0, 0, 0}, sF1[4] = {0, 0, 0, 0};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const long o = gc[v] * A.np;
                const float ll = (hasl && okc) ? (float)A.lamLt[o + il] : 0.0f;
                const float lr = (hasr && okc) ? (float)A.lamLt[o + ir] : 0.0f;
                sF1[v] = 0.25f * (-ll * ihl + lr * ihr);
                if (needF0) {
                    const float ml = (hasl && okc) ? (float)A.lamL[o + il] : 0.0f;
                    const float mr = (hasr && okc) ? (float)A.lamL[o + ir] : 0.0f;
                    sF0[v] = 0.25f * (-ml * ihl + mr * ihr);
                }
            }
            const float ih1 = A.ih1[a + G], ih2 = A.ih2[b + G];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                float Qv[2][4], Dn[2][4], D1[2][4], D2[2][4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float *x = st + (v * 4 + m) * ST_ROWS + ty * TX + tx;
                    const float *y = st + (v * 4 + 2 + m) * ST_ROWS + ty * TX + tx;
                    const float *z = st + (16 + v * 2 + m) * ST_ROWS + ty * TX + tx;
                    float vm, vp, dm, dp;
                    tan_val_der(x[0], x[TX], x[2 * TX], x[3 * TX], x[4 * TX], vm, vp, dm, dp);
                    Qv[0][v] = vm; Qv[1][v] = vp; D2[0][v] = dm; D2[1][v] = dp;
                    tan_val_direct(y[0], y[TX], y[2 * TX], y[3 * TX], y[4 * TX], vm, vp);
                    D1[0][v] = vm; D1[1][v] = vp;
                    tan_val_direct(z[0], z[TX], z[2 * TX], z[3 * TX], z[4 * TX], vm, vp);
                    Dn[0][v] = vm; Dn[1][v] = vp;
                }
                // the flux reverse at the two t2 Gauss points as one evaluation on
                // packed FP32 pairs (the points in the lanes)
                {
                    f2 q2[4], n2[4], a2[4], b2[4], s0[4], s1[4], qb[4], Dnb[4], D1b[4], D2b[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        q2[v] = f2(Qv[0][v], Qv[1][v]);
                        n2[v] = f2(Dn[0][v], Dn[1][v]);
                        a2[v] = f2(D1[0][v], D1[1][v]);
                        b2[v] = f2(D2[0][v], D2[1][v]);
                        s0[v] = f2(sF0[v]);
                        s1[v] = f2(sF1[v]);
                    }
                    Phys<f2> p2;
                    p2.lambda = f2(A.ph.lambda);
                    p2.theta = f2(A.ph.theta);
                    p2.mu = f2(A.ph.mu);
                    p2.off = f2(A.ph.off);
                    p2.sqlam = f2(A.ph.sqlam);
                    p2.kE = f2(A.ph.kE);
                    gk_flux_rev<f2>(p2, q2, n2, a2, b2, f2(ih1), f2(ih2), s0, s1, needF0, qb, Dnb, D1b, D2b);
#pragma unroll
                    for (int nn = 0; nn < 2; ++nn) {
                        float *gp = ga + (16 * (2 * m + nn)) * (TX * TY) + tid;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            gp[v * (TX * TY)] = nn ? qb[v].v.y : qb[v].v.x;
                            gp[(4 + v) * (TX * TY)] = nn ? Dnb[v].v.y : Dnb[v].v.x;
                            gp[(8 + v) * (TX * TY)] = nn ? D1b[v].v.y : D1b[v].v.x;
                            gp[(12 + v) * (TX * TY)] = nn ? D2b[v].v.y : D2b[v].v.x;
                        }
                    }
                }
            }
        } else {
#pragma unroll 4
            for (int j = 0; j < 64; ++j) ga[j * (TX * TY) + tid] = 0.0f;
        }
        __syncthreads();

        // RB: row r of the t1 pass is read by the faces bb = r - sx of the tile
        // with stencil index sx. A thread takes one array and one column: the
        // adjoints of the 8 faces of the column that the array's rows feed
        // sit in registers and the 12 rows are 5-tap sums of them (indices
        // and weights compile-time; the same terms in the same order as a
        // gather per row)
        for (int task = tid; task < 24 * TX; task += TX * TY) {
            const int arr = task / TX, c = task - arr * TX;
            int v, m, kind;   // kind 0: Q0 value rows, 1: t1-derivative rows, 2: normal-slope rows
            if (arr < 16) {
                v = arr >> 2;
                m = arr & 1;
                kind = (arr >> 1) & 1;
            } else {
                v = (arr - 16) >> 1;
                m = (arr - 16) & 1;
                kind = 2;
            }
            const int jq = kind == 0 ? v : (kind == 1 ? 8 + v : 4 + v);
            float X[TY][2], Y[TY][2];
#pragma unroll
            for (int bb = 0; bb < TY; ++bb)
#pragma unroll
                for (int nn = 0; nn < 2; ++nn) {
                    const float *g0 = ga + (16 * (2 * m + nn)) * (TX * TY) + bb * TX + c;
                    X[bb][nn] = g0[jq * (TX * TY)];
                    Y[bb][nn] = kind == 0 ? g0[(12 + v) * (TX * TY)] : 0.0f;
                }
            float *o = st + arr * ST_ROWS + c;
#pragma unroll
            for (int r = 0; r < SQ_H; ++r) {
                float acc = 0.0f;
#pragma unroll
                for (int sx = 0; sx < 5; ++sx) {
                    const int bb = r - sx;
                    if (bb < 0 || bb >= TY) continue;
#pragma unroll
                    for (int nn = 0; nn < 2; ++nn) {
                        acc += cWV32[nn][sx] * X[bb][nn];
                        if (kind == 0) acc += cWD32[nn][sx] * Y[bb][nn];
                    }
                }
                o[r * TX] = acc;
            }
        }
        __syncthreads();

        // RC: face-box column cc is read by the row columns c = cc - sx. A
        // thread takes one component, one row and 4 face-box columns cc0 ..
        // cc0+3: the 8 row columns cc0-4 .. cc0+3 of each array it needs come
        // by 128-bit loads (zero outside the tile), the 4 outputs are 5-tap
        // sums of them and leave by one 128-bit store
        float *out = A.part + (long)t * kPartN;
        constexpr int NG = SQ_W / 4;   // 9 groups of 4 columns
        for (int task = tid; task < 8 * SQ_H * NG; task += TX * TY) {
            const int j = task / (SQ_H * NG), rem = task - j * (SQ_H * NG), r = rem / NG, gq = rem - r * NG;
            const int cc0 = 4 * gq;
            const int na = j < 4 ? 4 : 2;
            int arrs[4];
            if (j < 4) {
                arrs[0] = j * 4; arrs[1] = j * 4 + 1; arrs[2] = j * 4 + 2; arrs[3] = j * 4 + 3;
            } else {
                arrs[0] = 16 + (j - 4) * 2; arrs[1] = arrs[0] + 1; arrs[2] = arrs[3] = arrs[0];
            }
            float Z[4][8];   // per array, row columns cc0-4 .. cc0+3
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float *rowp = st + arrs[q] * ST_ROWS + r * TX;
                const float4 lo4 = (q < na && cc0 >= 4) ? *reinterpret_cast<const float4 *>(rowp + cc0 - 4)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 hi4 = (q < na && cc0 < TX) ? *reinterpret_cast<const float4 *>(rowp + cc0)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                Z[q][0] = lo4.x; Z[q][1] = lo4.y; Z[q][2] = lo4.z; Z[q][3] = lo4.w;
                Z[q][4] = hi4.x; Z[q][5] = hi4.y; Z[q][6] = hi4.z; Z[q][7] = hi4.w;
            }
            float res[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float acc = 0.0f;
#pragma unroll
                for (int sx = 0; sx < 5; ++sx) {
                    const int k = 4 + i - sx;   // row column cc0 + i - sx
                    if (cc0 + i - sx < 0 || cc0 + i - sx >= TX) continue;
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        if (j < 4)
                            acc += cWV32[m][sx] * Z[m][k] + cWD32[m][sx] * Z[2 + m][k];
                        else
                            acc += cWV32[m][sx] * Z[m][k];
                    }
                }
                res[i] = acc;
            }
            *reinterpret_cast<float4 *>(out + (j * SQ_H + r) * SQ_W + cc0) = make_float4(res[0], res[1], res[2], res[3]);
        }
        __syncthreads();   // the buffers are free for the next tile
    }
}

// Face-box adjoints of direction d (the layout of the forward's face box)
// from the tile partials: face (f, a', b') of the extended box lies in the
// tangential halo of at most two tiles along each axis; their partials are
// added in tile order.
__global__ void __launch_bounds__(256) sum_partials32_kernel(const float *part, float *lamFQ, long nfq, int e1p,
                                                             int n1, int n2)
{
    const int ap = (int)(blockIdx.x * TX + threadIdx.x) - 2, bp = (int)(blockIdx.y * TY + threadIdx.y) - 2;
    const int f = blockIdx.z;
    if (ap >= n1 + 2 || bp >= n2 + 2) return;
    const int NA = (n1 + TX - 1) / TX, NB = (n2 + TY - 1) / TY;
    const int ta1 = (ap + 2) / TX, tb1 = (bp + 2) / TY;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int ta = ta1 - 1; ta <= ta1; ++ta) {
        const int cc = ap + 2 - ta * TX;
        if (ta < 0 || ta >= NA || cc < 0 || cc >= SQ_W) continue;
        for (int tb = tb1 - 1; tb <= tb1; ++tb) {
            const int r = bp + 2 - tb * TY;
            if (tb < 0 || tb >= NB || r < 0 || r >= SQ_H) continue;
            const float *p = part + (long)(ta + NA * (tb + NB * (long)f)) * kPartN + r * SQ_W + cc;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += p[j * (SQ_H * SQ_W)];
        }
    }
    const long o = ((long)f * (n2 + 4) + (bp + 2)) * e1p + (ap + 2);
    if (!in_bounds(o, nfq)) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) lamFQ[j * nfq + o] = acc[j];
}

// Ghost adjoint of one (axis, side, layer): the ghost's adjoint goes to its
// source cell and is cleared.
struct GhostRevArgs {
    const double *A;  // forward working array
    double *lamA;
    double *uinf_part;
    int n[3], P[3];
    long np;
    int d, e1, e2, lo1, lo2, len1, len2, s, bc;
    long uinf_layer;   // stride of uinf_part between layers
    double csound, uin[3];
};

// One (axis, side): the layers l = G .. 1 in turn, each thread one position
// of the side (the sources are interior cells, so a thread's layers are its
// own and keep the order of a sweep per layer).
__global__ void __launch_bounds__(256) ghost_rev_kernel(GhostRevArgs A)
{
    const int a = A.lo1 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int b = A.lo2 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    if (a >= A.lo1 + A.len1 || b >= A.lo2 + A.len2) return;
    const int d = A.d, nd = A.n[d], s = A.s, bc = A.bc;
    for (int l = G; l >= 1; --l) {
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
        const long ig = lin(A.P[0], A.P[1], cg[0], cg[1], cg[2]), is = lin(A.P[0], A.P[1], cs[0], cs[1], cs[2]);
        if (!in_bounds(ig, A.np) || !in_bounds(is, A.np)) continue;
        double lg[4];
        for (int v = 0; v < 4; ++v) {
            lg[v] = A.lamA[v * A.np + ig];
            A.lamA[v * A.np + ig] = 0.0;
        }
        double add[4] = {lg[0], lg[1], lg[2], lg[3]};
        double gu = 0.0;
        if (bc == GKS_BC_NOSLIP) {
            add[1] = -lg[1]; add[2] = -lg[2]; add[3] = -lg[3];
        } else if (bc == GKS_BC_SLIP) {
            add[1 + d] = -lg[1 + d];
        } else if (bc == GKS_BC_INFLOW) {
            const double r1 = A.A[is], un1 = A.A[(1 + d) * A.np + is] / r1;
            const double sg = s == 0 ? 1.0 : -1.0;
            const double x = sg * (A.uin[d] - un1) / A.csound;
            const double ex = exp(x);
            const double rg = r1 * ex;
            const double rgb = lg[0] + lg[1] * A.uin[0] + lg[2] * A.uin[1] + lg[3] * A.uin[2];
            add[0] = rgb * ex * (1.0 + sg * un1 / A.csound);
            add[1] = add[2] = add[3] = 0.0;
            add[1 + d] = -rgb * sg * ex / A.csound;
            // sensitivity to the inflow speed U_inf = u_in[0]
            gu = lg[1] * rg + (d == 0 ? rgb * r1 * ex * sg / A.csound : 0.0);
        }
        for (int v = 0; v < 4; ++v) A.lamA[v * A.np + is] += add[v];
        if (bc == GKS_BC_INFLOW)
            A.uinf_part[(long)(l - 1) * A.uinf_layer + (long)(b - A.lo2) * A.len1 + (a - A.lo1)] = gu;
    }
}

// Fixed-order two-pass sum of x[0..n) added to *acc: block b of kRedBlocks
// sums its contiguous chunk (thread-strided, then a shared-memory tree) into
// part[b]; one block then sums the parts the same way.
constexpr int kRedBlocks = 256;

__global__ void __launch_bounds__(256) reduce_part_kernel(const double *x, long n, double *part)
{
    __shared__ double sh[256];
    const long chunk = (n + kRedBlocks - 1) / kRedBlocks, i0 = blockIdx.x * chunk;
    const long i1 = i0 + chunk < n ? i0 + chunk : n;
    double s = 0.0;
    for (long i = i0 + threadIdx.x; i < i1; i += 256) s += x[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) reduce_final_kernel(const double *part, double *acc)
{
    __shared__ double sh[256];
    sh[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += sh[0];
}

// Stage combinations, reversed (interior cells, padded indexing).
//   stage 2: W' = P + dt^2/3 Lt(W*):     lamLt = dt^2/3 lamP
//   stage 1: W* = W + dt/2 L + dt^2/8 Lt, P = W + dt L + dt^2/6 Lt:
//            lamW = lamWs + lamP, lamL = dt/2 lamWs + dt lamP,
//            lamLt = dt^2/8 lamWs + dt^2/6 lamP
__global__ void __launch_bounds__(256) rev_update_kernel(int stage, const double *lamWs, const double *lamP,
                                                         double *lamW, double *lamL, double *lamLt, double dt,
                                                         long np, int nx, int ny, int P0, int P1)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long l = lin(P0, P1, i, j, k);
    for (int v = 0; v < 4; ++v) {
        const long o = v * np + l;
        if (stage == 2) {
            lamLt[o] = dt * dt / 3.0 * lamP[o];
        } else {
            const double ws = lamWs[o], p = lamP[o];
            lamW[o] = ws + p;
            lamL[o] = 0.5 * dt * ws + dt * p;
            lamLt[o] = 0.125 * dt * dt * ws + dt * dt / 6.0 * p;
        }
    }
}

// ---------------------------------------------------------------- ALM adjoint

struct AlmAdjArgs {
    int P[3], n[3];
    long np;
    double x0[3], h[3];
    const double *Wp;    // state the loads were sampled from
    double *lam;         // adjoint of the state after forcing (in: lambda'', out: lambda')
    RotorDev r;
    double *pts;         // 8 per point
    double dt, power_seed, t;
};

__device__ __forceinline__ double centre_d(const AlmAdjArgs &A, int d, int i)
{
    return __dadd_rn(A.x0[d], __dmul_rn((double)i + 0.5, A.h[d]));
}

__device__ __forceinline__ double dist3(double dx, double dy, double dz)
{
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

// mu_p = d J / d (F_x, F_th)_p from the projection: -dt sum_cells lambda_m . e eta
__global__ void __launch_bounds__(256) alm_interp_adj_kernel(AlmAdjArgs A)
{
    __shared__ double sx[256], stt[256];
    const int q = blockIdx.x;
    const RotorDev &r = A.r;
    const int b = q / r.np;
    const double X[3] = {r.X[3 * q], r.X[3 * q + 1], r.X[3 * q + 2]};
    const double e1 = r.et[2 * b], e2 = r.et[2 * b + 1];
    const double cut = 3.0 * r.eps, norm = 1.0 / (r.eps * r.eps * r.eps * pow(kPi, 1.5));
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = (int)floor((X[d] - cut - A.x0[d]) / A.h[d] - 0.5) - 1;
        hi[d] = (int)ceil((X[d] + cut - A.x0[d]) / A.h[d] - 0.5) + 1;
        if (lo[d] < r.box[d][0]) lo[d] = r.box[d][0];
        if (hi[d] > r.box[d][1]) hi[d] = r.box[d][1];
    }
    const int bx = hi[0] - lo[0] + 1, by = hi[1] - lo[1] + 1, bz = hi[2] - lo[2] + 1;
    double ax = 0.0, at = 0.0;
    const long nc = (bx > 0 && by > 0 && bz > 0) ? (long)bx * by * bz : 0;
    for (long c = threadIdx.x; c < nc; c += blockDim.x) {
        const int i = lo[0] + (int)(c % bx), j = lo[1] + (int)((c / bx) % by), k = lo[2] + (int)(c / ((long)bx * by));
        const double rr = dist3(centre_d(A, 0, i) - X[0], centre_d(A, 1, j) - X[1], centre_d(A, 2, k) - X[2]);
        if (rr > cut) continue;
        const double eta = exp(-(rr / r.eps) * (rr / r.eps)) * norm;
        const long l = lin(A.P[0], A.P[1], i, j, k);
        ax += A.lam[A.np + l] * eta;
        at += (A.lam[2 * A.np + l] * e1 + A.lam[3 * A.np + l] * e2) * eta;
    }
    sx[threadIdx.x] = ax;
    stt[threadIdx.x] = at;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sx[threadIdx.x] += sx[threadIdx.x + w];
            stt[threadIdx.x] += stt[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.pts[8 * q + 0] = -A.dt * sx[0];
        A.pts[8 * q + 1] = -A.dt * stt[0];
    }
}

__device__ bool trilinear_w(const AlmAdjArgs &A, const double X[3], int i0[3], double fr[3])
{
    for (int d = 0; d < 3; ++d) {
        const double s = (X[d] - A.x0[d]) / A.h[d] - 0.5;
        const double fl = floor(s);
        i0[d] = (int)fl;
        fr[d] = s - fl;
        if (i0[d] < 0 || i0[d] + 1 > A.n[d] - 1) {
            if (A.n[d] == 1 && s >= -0.5 && s <= 0.5) {
                i0[d] = 0;
                fr[d] = 0.0;
                continue;
            }
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ double cd_of(double a) { return 0.01 + 0.02 * a * a; }

// Tip factor F(phi) = (2/pi) acos(exp(-x)), x = g1 N (R - r) / (2 r |sin phi|)
// (the same expression as the forward) and dF/dphi = (2/pi) e^-x x' /
// sqrt(1 - e^-2x) with x' = -x cot phi; F = 0 with zero slope at and beyond
// the tip, zero slope where e^-x underflows (sin phi -> 0, F -> 1).
__device__ __forceinline__ void tip_factor_d(double g1, int nb, double R, double r, double phi, double &F,
                                             double &dF)
{
    F = 0.0;
    dF = 0.0;
    if (r >= R) return;
    const double sp = sin(phi);
    const double x = g1 * nb * (R - r) / (2.0 * r * fabs(sp));
    const double e = exp(-x);
    F = (2.0 / kPi) * acos(e);
    if (e > 0.0) dF = (2.0 / kPi) * e * (-x * cos(phi) / sp) / sqrt(-expm1(-2.0 * x));
}

// Reverse of the point loads: gradient of the force scales (this step), the
// power seed, and the adjoint of the sampled velocity.
__global__ void __launch_bounds__(256) alm_loads_adj_kernel(AlmAdjArgs A)
{
    const RotorDev &r = A.r;
    const int npts = r.nb * r.np;
    for (int q = threadIdx.x; q < npts; q += blockDim.x) {
        const int b = q / r.np, p = q - b * r.np;
        const double th = r.az0 + r.omega * A.t + 2.0 * kPi * b / r.nb;
        const double cth = cos(th), sth = sin(th);
        const double rr = r.r[p];
        const double X[3] = {r.hub[0], r.hub[1] + rr * cth, r.hub[2] + rr * sth};
        int i0[3];
        double fr[3];
        double Ub[3] = {0, 0, 0}, gs = 0.0;
        if (trilinear_w(A, X, i0, fr)) {
            double U[3] = {0, 0, 0};
            for (int c = 0; c < 8; ++c) {
                const int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
                const double w = (di ? fr[0] : 1.0 - fr[0]) * (dj ? fr[1] : 1.0 - fr[1]) * (dk ? fr[2] : 1.0 - fr[2]);
                if (w == 0.0) continue;
                const int ii = A.n[0] == 1 ? 0 : i0[0] + di, jj = A.n[1] == 1 ? 0 : i0[1] + dj;
                const int kk = A.n[2] == 1 ? 0 : i0[2] + dk;
                const long l = lin(A.P[0], A.P[1], ii, jj, kk);
                const double rho = A.Wp[l];
                U[0] += w * A.Wp[A.np + l] / rho;
                U[1] += w * A.Wp[2 * A.np + l] / rho;
                U[2] += w * A.Wp[3 * A.np + l] / rho;
            }
            // velocity correction (one pass with C_D of the uncorrected angle)
            const double ux0 = U[0], ut0 = -sth * U[1] + cth * U[2];
            const double wr = r.omega * rr;
            double fac = 1.0, phi0 = 0.0;
            if (r.correction) {
                phi0 = atan2(ux0, wr - ut0);
                const double cd0 = cd_of(phi0 - r.twist[p]);
                fac = 1.0 / (1.0 - cd0 * r.chord[p] / (4.0 * sqrt(kPi) * r.eps));
            }
            const double ux = ux0 * fac, ut = ut0 * fac;
            const double av = ux, bv = wr - ut;
            const double phi = atan2(av, bv), al = phi - r.twist[p];
            const double urel2 = av * av + bv * bv;
            const double qk = 0.5 * r.rho_inf * r.chord[p] * r.width[p];
            const double qd = qk * urel2;
            const double clr = 2.0 * kPi * sin(al);
            const double cl = clr > 1.4 ? 1.4 : (clr < -1.4 ? -1.4 : clr);
            const double dcl = (clr > 1.4 || clr < -1.4) ? 0.0 : 2.0 * kPi * cos(al);
            const double cd = cd_of(al);
            const double Lf = qd * cl, Df = qd * cd;
            const double cp = cos(phi), sp = sin(phi);
            const double fx = Lf * cp + Df * sp, ft = Lf * sp - Df * cp;
            // tip factors of the axial and tangential loads
            double tx = 1.0, tt = 1.0, dtx = 0.0, dtt = 0.0;
            if (r.tip) {
                tip_factor_d(r.tip_g[0], r.nb, r.radius, rr, phi, tx, dtx);
                tip_factor_d(r.tip_g[1], r.nb, r.radius, rr, phi, tt, dtt);
            }
            const double s = r.scale[q];
            const double mux = A.pts[8 * q + 0];
            const double mut = A.pts[8 * q + 1] + A.power_seed * r.omega * rr;
            gs = mux * tx * fx + mut * tt * ft;
            const double fxb = s * tx * mux, ftb = s * tt * mut;
            const double Lb = fxb * cp + ftb * sp, Db = fxb * sp - ftb * cp;
            double phib = fxb * (-Lf * sp + Df * cp) + ftb * (Lf * cp + Df * sp) +
                          s * (mux * fx * dtx + mut * ft * dtt);
            const double qdb = Lb * cl + Db * cd;
            const double alb = Lb * qd * dcl + Db * qd * 0.04 * al;
            phib += alb;
            const double u2b = qdb * qk;
            const double den = urel2 > 0.0 ? urel2 : 1.0;
            const double ab = phib * bv / den + u2b * 2.0 * av;
            const double bb = -phib * av / den + u2b * 2.0 * bv;
            double uxb = ab, utb = -bb;
            if (r.correction) {
                // ux = fac ux0, ut = fac ut0, fac = 1 / (1 - k C_D(phi0 - twist)),
                // dfac/dC_D = k fac^2, phi0 = atan2(ux0, wr - ut0)
                const double k = r.chord[p] / (4.0 * sqrt(kPi) * r.eps);
                const double facb = uxb * ux0 + utb * ut0;
                const double phi0b = facb * k * fac * fac * 0.04 * (phi0 - r.twist[p]);
                const double b0 = wr - ut0, d0 = ux0 * ux0 + b0 * b0;
                const double den0 = d0 > 0.0 ? d0 : 1.0;
                uxb = fac * uxb + phi0b * b0 / den0;
                utb = fac * utb + phi0b * ux0 / den0;
            }
            Ub[0] = uxb;
            Ub[1] = -sth * utb;
            Ub[2] = cth * utb;
        }
        A.pts[8 * q + 2] = gs;
        A.pts[8 * q + 3] = Ub[0];
        A.pts[8 * q + 4] = Ub[1];
        A.pts[8 * q + 5] = Ub[2];
    }
}

// Reverse of the trilinear sampling. One thread per point forms the
// adjoints its 8 corner cells receive (cell index and 4 values per corner,
// zero weight -> index -1) in ptc/ptl; one thread then adds them in point
// and corner order (deterministic; points can share cells).
__global__ void __launch_bounds__(256) alm_sample_adj_kernel(AlmAdjArgs A, double *ptc, long *ptl)
{
    const RotorDev &r = A.r;
    const int npts = r.nb * r.np;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npts) return;
    for (int c = 0; c < 8; ++c) ptl[8 * q + c] = -1;
    const int b = q / r.np, p = q - b * r.np;
    const double th = r.az0 + r.omega * A.t + 2.0 * kPi * b / r.nb;
    const double rr = r.r[p];
    const double X[3] = {r.hub[0], r.hub[1] + rr * cos(th), r.hub[2] + rr * sin(th)};
    int i0[3];
    double fr[3];
    if (!trilinear_w(A, X, i0, fr)) return;
    const double Ub[3] = {A.pts[8 * q + 3], A.pts[8 * q + 4], A.pts[8 * q + 5]};
    for (int c = 0; c < 8; ++c) {
        const int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        const double w = (di ? fr[0] : 1.0 - fr[0]) * (dj ? fr[1] : 1.0 - fr[1]) * (dk ? fr[2] : 1.0 - fr[2]);
        if (w == 0.0) continue;
        const int ii = A.n[0] == 1 ? 0 : i0[0] + di, jj = A.n[1] == 1 ? 0 : i0[1] + dj;
        const int kk = A.n[2] == 1 ? 0 : i0[2] + dk;
        const long l = lin(A.P[0], A.P[1], ii, jj, kk);
        const double rho = A.Wp[l];
        double dot = 0.0;
        for (int v = 0; v < 3; ++v) {
            ptc[32 * q + 4 * c + 1 + v] = w * Ub[v] / rho;
            dot += Ub[v] * A.Wp[(1 + v) * A.np + l];
        }
        ptc[32 * q + 4 * c] = -w * dot / (rho * rho);
        ptl[8 * q + c] = l;
    }
}

// The sampling adjoints added to their cells. Entries e = 8 q + c (point q,
// corner c) name a cell (or -1 for a zero weight); points share cells. One
// block sorts the (cell, entry) keys (bitonic, in shared memory), so that
// each cell's entries sit together in entry order, and the first thread of
// each cell adds their sum: deterministic, and no two threads write a cell.
// More than kSampleSort entries take the sequential kernel below.
constexpr int kSampleSort = 2048;

__global__ void __launch_bounds__(1024) alm_sample_add_kernel(AlmAdjArgs A, const double *ptc, const long *ptl)
{
    __shared__ unsigned long long key[kSampleSort];
    constexpr unsigned long long kNone = ~0ull;
    const int n = 8 * A.r.nb * A.r.np;
    for (int i = threadIdx.x; i < kSampleSort; i += blockDim.x) {
        const long l = i < n ? ptl[i] : -1;
        key[i] = l < 0 ? kNone : ((unsigned long long)l << 12) | (unsigned long long)i;
    }
    __syncthreads();
    for (int k = 2; k <= kSampleSort; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < kSampleSort; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long a = key[i], b = key[p];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long ki = key[i];
        if (ki == kNone) continue;
        const unsigned long long cell = ki >> 12;
        if (i > 0 && (key[i - 1] >> 12) == cell) continue;
        double acc[4] = {0, 0, 0, 0};
        for (int j = i; j < n && key[j] != kNone && (key[j] >> 12) == cell; ++j) {
            const long e = (long)(key[j] & 4095ull);
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[v] += ptc[4 * e + v];
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) A.lam[v * A.np + (long)cell] += acc[v];
    }
}

__global__ void alm_sample_add_serial_kernel(AlmAdjArgs A, const double *ptc, const long *ptl)
{
    const int npts = A.r.nb * A.r.np;
    for (int q = 0; q < npts; ++q)
        for (int c = 0; c < 8; ++c) {
            const long l = ptl[8 * q + c];
            if (l < 0) continue;
            for (int v = 0; v < 4; ++v) A.lam[v * A.np + l] += ptc[32 * q + 4 * c + v];
        }
}

// S^T: adjoint of the spatial operator of working array Aw (ghost-filled),
// for lamL (may be null) and lamLt; result accumulated into w.lamA.
template <typename T>
void spatial_adjoint(const Ctx &c, const AdjWork &w, const double *Aw, void *const gp[3],
                     const double *lamL, const double *lamLt)
{
    const Phys<double> ph = make_phys<double>(c);
    constexpr bool f32 = sizeof(T) == 4;
    float *Ahi = (float *)w.Asplit, *Alo = Ahi + 4 * c.np;
    if (f32) {
        const long n = 4 * c.np, nb = (n + 255) / 256;
        split_kernel<<<(int)(nb < 16L * sm_count() ? nb : 16L * sm_count()), 256, 0, c.stream>>>(Aw, Ahi, Alo, n);
    }
    for (int d = 0; d < 3; ++d) {
        const int t1 = tan1(d), t2 = tan2(d);
        RevArgs R;
        R.A = Aw;
        R.Ahi = Ahi;
        R.Alo = Alo;
        R.nfq = c.nfq;
        R.e1p = c.e1p[d];
        R.lamL = lamL;
        R.lamLt = lamLt;
        R.lamG = gp[d];   // Gauss-point inputs of this direction (read only)
        R.lamGa = w.lamGa;
        R.nG = w.nG;
        R.lamR = w.lamR;
        R.nR = w.nR;
        R.lamFQ = w.lamFQ;
        R.lamC = w.lamC;
        R.lamA = w.lamA;
        R.ihd = (const double *)c.ih[d];
        R.ih1 = (const double *)c.ih[t1];
        R.ih2 = (const double *)c.ih[t2];
        R.ihf = (const double *)c.ihf[d];
        for (int e = 0; e < 3; ++e) {
            R.n[e] = c.n[e];
            R.P[e] = c.P[e];
        }
        R.d = d;
        R.t1 = t1;
        R.t2 = t2;
        R.nd = c.n[d];
        R.n1 = c.n[t1];
        R.n2 = c.n[t2];
        R.np = c.np;
        R.ph = ph;
        const dim3 blk(32, 8);
        const int nf = c.n[d] + 1;
        rev_flux_kernel<T><<<dim3((R.n1 + 31) / 32, (R.n2 + kRevFluxB - 1) / kRevFluxB, nf), blk, 0, c.stream>>>(R);
        rev_t2_kernel<T><<<dim3((R.n1 + 31) / 32, (R.n2 + 4 + kRevT2 - 1) / kRevT2, nf), blk, 0, c.stream>>>(R);
        rev_t1_kernel<T><<<dim3((R.n1 + 4 + 31) / 32, (R.n2 + 4 + 7) / 8, nf), blk, 0, c.stream>>>(R);
        const dim3 gfs((R.n1 + 4 + 31) / 32, (R.n2 + 4 + 7) / 8, (nf + kRevMarch - 1) / kRevMarch);
        if (f32)
            rev_face_state32_kernel<true><<<gfs, blk, 0, c.stream>>>(R);
        else
            rev_face_state_kernel<<<gfs, blk, 0, c.stream>>>(R);
        rev_gather_cells_kernel<T><<<dim3((R.n1 + 4 + 31) / 32, (R.n2 + 4 + 7) / 8, R.nd + 2 * G), blk, 0,
                                     c.stream>>>(R);
    }
}

// S^T of an FP32C grid through the fused reverse: per direction the forward
// face boxes from the FP32 working array A32 (as the forward read it), RA-RC
// in one pass over the tiles, the partials added per face, then RD on the
// FP32 cells and RE. c32 is the grid's own context (FP32 widths, the density
// offset, the face-box buffer and its TMA maps); cw the reverse's context.
void spatial_adjoint_fused32(const Ctx &cw, const AdjWork &w, const float *A32, const double *lamL,
                             const double *lamLt)
{
    const Ctx &c = *w.c32;
    const Phys<float> ph = make_phys<float>(c);
    const dim3 blk(TX, TY);
    const size_t smem = rev_tile32_smem_bytes();
    static int grid_blocks = 0;
    if (!grid_blocks) {
        int per = 0;
        cudaFuncSetAttribute(rev_tile32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rev_tile32_kernel, TX * TY, smem);
        grid_blocks = (per > 0 ? per : 1) * sm_count();
    }
    for (int d = 0; d < 3; ++d) {
        const int t1 = tan1(d), t2 = tan2(d);
        launch_face_state32(c, d, A32);
        Rev32Args Q;
        Q.lamL = lamL;
        Q.lamLt = lamLt;
        Q.ihd = (const float *)c.ih[d];
        Q.ih1 = (const float *)c.ih[t1];
        Q.ih2 = (const float *)c.ih[t2];
        Q.part = w.part;
        Q.n1 = c.n[t1];
        Q.n2 = c.n[t2];
        Q.nf = c.n[d] + 1;
        Q.nd = c.n[d];
        Q.d = d;
        Q.t1 = t1;
        Q.t2 = t2;
        const long stride[3] = {1, (long)c.P[0], (long)c.P[0] * c.P[1]};
        Q.sd = stride[d];
        Q.s1 = stride[t1];
        Q.s2 = stride[t2];
        Q.base = G * (stride[0] + stride[1] + stride[2]);
        Q.np = c.np;
        Q.ph = ph;
        Q.scal = w.sc;
        const long ntiles = (long)((Q.n1 + TX - 1) / TX) * ((Q.n2 + TY - 1) / TY) * Q.nf;
        const int grid = (int)(ntiles < grid_blocks ? ntiles : grid_blocks);
        rev_tile32_kernel<<<grid, blk, smem, c.stream>>>(c.tmap[d], Q);
        sum_partials32_kernel<<<dim3((Q.n1 + 4 + TX - 1) / TX, (Q.n2 + 4 + TY - 1) / TY, Q.nf), blk, 0, c.stream>>>(
            w.part, (float *)w.lamFQ, c.nfq, c.e1p[d], Q.n1, Q.n2);
        // RD on the FP32 cells (density as rho - off, the forward's offset) and RE
        RevArgs R;
        R.A = nullptr;
        R.Ahi = A32;
        R.Alo = nullptr;
        R.nfq = c.nfq;
        R.e1p = c.e1p[d];
        R.lamL = lamL;
        R.lamLt = lamLt;
        R.lamFQ = w.lamFQ;
        R.lamC = w.lamC;
        R.lamA = w.lamA;
        R.ihf = (const double *)cw.ihf[d];
        for (int e = 0; e < 3; ++e) {
            R.n[e] = c.n[e];
            R.P[e] = c.P[e];
        }
        R.d = d;
        R.t1 = t1;
        R.t2 = t2;
        R.nd = c.n[d];
        R.n1 = c.n[t1];
        R.n2 = c.n[t2];
        R.np = c.np;
        R.ph = make_phys<double>(c);
        const int nf = c.n[d] + 1;
        const dim3 gfs((R.n1 + 4 + 31) / 32, (R.n2 + 4 + 7) / 8, (nf + kRevMarch - 1) / kRevMarch);
        (void)gfs;
        rev_face_cells32_kernel<<<dim3((R.n1 + 4 + 31) / 32, (R.n2 + 4 + 7) / 8,
                                       (R.nd + 2 * G + kRevCells - 1) / kRevCells), blk, 0, c.stream>>>(R);
    }
}

// Adjoint of the ghost fill of working array Aw: axes z, y, x (reverse of
// the forward sweep), each side and layer in turn.
void ghost_adjoint(const Ctx &c, const AdjWork &w, const double *Aw)
{
    cudaMemsetAsync(w.uinf_part, 0, sizeof(double) * w.nuinf, c.stream);
    for (int d = 2; d >= 0; --d) {
        GhostRevArgs A;
        A.A = Aw;
        A.lamA = w.lamA;
        for (int e = 0; e < 3; ++e) {
            A.n[e] = c.n[e];
            A.P[e] = c.P[e];
        }
        A.np = c.np;
        A.d = d;
        A.e1 = tan1(d);
        A.e2 = tan2(d);
        A.lo1 = A.e1 < d ? -G : 0;
        A.len1 = A.e1 < d ? c.n[A.e1] + 2 * G : c.n[A.e1];
        A.lo2 = A.e2 < d ? -G : 0;
        A.len2 = A.e2 < d ? c.n[A.e2] + 2 * G : c.n[A.e2];
        A.csound = c.csound;
        for (int e = 0; e < 3; ++e) A.uin[e] = c.inflow[1 + e];
        for (int s = 0; s < 2; ++s) {
            A.s = s;
            A.bc = c.bc[d][s];
            A.uinf_layer = w.nuinf / (6 * G);
            A.uinf_part = w.uinf_part + (long)((d * 2 + s) * G) * A.uinf_layer;
            ghost_rev_kernel<<<dim3((A.len1 + 31) / 32, (A.len2 + 7) / 8, 1), dim3(32, 8), 0, c.stream>>>(A);
        }
    }
    static_assert(kRedBlocks == 256, "one part per thread of the final pass");
    reduce_part_kernel<<<kRedBlocks, 256, 0, c.stream>>>(w.uinf_part, w.nuinf, w.red);
    reduce_final_kernel<<<1, 256, 0, c.stream>>>(w.red, w.scal);
}

__global__ void __launch_bounds__(256) add_interior_kernel(double *dst, const double *src, long np, int nx, int ny,
                                                           int P0, int P1)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long l = lin(P0, P1, i, j, k);
    for (int v = 0; v < 4; ++v) dst[v * np + l] += src[v * np + l];
}

// Reverse of the direct-forcing iterations of one immersed body with a fixed
// iteration count N (Sec. 3.2, Eq. (ibm-1)): per box cell with Vbar > 0 each
// iteration is m <- m + rho phi (vbar - m / rho) = (1 - phi) m + phi rho vbar
// (density unchanged), so m_N = q m + (1 - q) rho vbar with q = (1 - phi)^N,
// and lambda_m <- q lambda_m, lambda_rho += (1 - q) sum_d vbar_d lambda_m_d.
__global__ void __launch_bounds__(256) ibm_adj_kernel(double *lam, long np, int P0, int P1, BodyDev b)
{
    const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (c >= b.nbox) return;
    if (!(b.Vbar[c] > 0.0)) return;
    const int bx = b.box[0][1] - b.box[0][0] + 1, by = b.box[1][1] - b.box[1][0] + 1;
    const int i = b.box[0][0] + (int)(c % bx);
    const int j = b.box[1][0] + (int)((c / bx) % by);
    const int k = b.box[2][0] + (int)(c / ((long)bx * by));
    const long l = lin(P0, P1, i, j, k);
    double q = 1.0;
    for (int s = 0; s < b.niter; ++s) q *= 1.0 - b.phi[c];
    double lr = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double lm = lam[(1 + d) * np + l];
        lam[(1 + d) * np + l] = q * lm;
        lr += (1.0 - q) * b.vbar[3 * c + d] * lm;
    }
    lam[l] += lr;
}

}  // namespace

namespace {
struct Carver {
    uintptr_t b0;
    size_t o = 0;
    double *take(size_t n)
    {
        double *p = (double *)(b0 + o);
        o += (n * sizeof(double) + 255) & ~(size_t)255;
        return p;
    }
};
}  // namespace

size_t adjoint_tape_carve(const Ctx &c, int gp_bytes, void *base, AdjWork *w)
{
    Carver k{(uintptr_t)base};
    w->gp_bytes = gp_bytes;
    const long np4 = 4 * c.np;
    w->hdr = k.take(kTapeHeader);
    w->A0 = k.take(np4);
    w->Ws = k.take(np4);
    w->Wp = k.take(np4);
    long nG = 0;
    for (int d = 0; d < 3; ++d) nG = std::max(nG, (long)(c.n[d] + 1) * c.n[tan1(d)] * c.n[tan2(d)]);
    w->nG = nG;
    if (c.prec == GKS_FP32C) {
        // the reverse recomputes the face boxes and Gauss-point inputs from
        // the FP32 working arrays (the fused reverse): no Gauss-point tape
        w->A0f = (float *)k.take(np4 / 2);
        w->Wsf = (float *)k.take(np4 / 2);
        for (int st = 0; st < 2; ++st)
            for (int d = 0; d < 3; ++d) w->gps[st][d] = nullptr;
        return k.o;
    }
    for (int st = 0; st < 2; ++st)
        for (int d = 0; d < 3; ++d) {
            w->gps[st][d] = k.take(64 * nG * gp_bytes / 8);
        }
    return k.o;
}

size_t adjoint_scratch_carve(const Ctx &c, long npts_total, void *base, AdjWork *w)
{
    Carver k{(uintptr_t)base};
    const long np4 = 4 * c.np;
    w->lamA = k.take(np4);
    w->lamW = k.take(np4);
    w->lamP = k.take(np4);
    w->lamL = k.take(np4);
    w->lamLt = k.take(np4);
    long nR = 0, maxsurf = 0;
    for (int d = 0; d < 3; ++d) {
        const int t1 = tan1(d), t2 = tan2(d);
        nR = std::max(nR, (long)(c.n[d] + 1) * (c.n[t2] + 4) * c.n[t1]);
        const long l1 = t1 < d ? c.n[t1] + 2 * G : c.n[t1];
        const long l2 = t2 < d ? c.n[t2] + 2 * G : c.n[t2];
        maxsurf = std::max(maxsurf, l1 * l2);
    }
    w->nR = nR;
    w->lamFQ = k.take(8 * c.nfq);
    w->lamC = k.take(24 * c.nfq);
    if (c.prec == GKS_FP32C) {
        // the fused reverse: tile partials instead of Gauss-point and row adjoints
        long np = 0;
        for (int d = 0; d < 3; ++d)
            np = std::max(np, (long)((c.n[tan1(d)] + TX - 1) / TX) * ((c.n[tan2(d)] + TY - 1) / TY) * (c.n[d] + 1));
        w->part = (float *)k.take((np * kPartN + 1) / 2);
        w->lamR = w->lamGa = w->Asplit = nullptr;
    } else {
        w->lamR = k.take(24 * nR);
        long nG = 0;
        for (int d = 0; d < 3; ++d) nG = std::max(nG, (long)(c.n[d] + 1) * c.n[tan1(d)] * c.n[tan2(d)]);
        w->lamGa = k.take(64 * nG);     // Gauss-point adjoints of one direction (double or float)
        w->Asplit = k.take(4 * c.np);   // 8 np floats: hi, lo
    }
    w->nuinf = 3 * 2 * G * maxsurf;
    w->uinf_part = k.take(w->nuinf);
    w->red = k.take(kRedBlocks);
    const long np = npts_total > 0 ? npts_total : 1;
    w->pts = k.take(8 * np);
    w->ptc = k.take(32 * np);
    w->ptl = k.take(8 * np);
    w->scal = k.take(8);
    w->sc = (Scalars *)k.take((sizeof(Scalars) + 7) / 8);
    for (int d = 0; d < 3; ++d) {
        w->ih64[d] = k.take(c.P[d]);
        w->ihf64[d] = k.take(c.n[d] + 1);
    }
    return k.o;
}

size_t adjoint_carve(const Ctx &c, long npts_total, int gp_bytes, void *base, AdjWork *w)
{
    const size_t tb = adjoint_tape_carve(c, gp_bytes, base, w);
    return tb + adjoint_scratch_carve(c, npts_total, base ? (void *)((uintptr_t)base + tb) : (void *)tb, w);
}

size_t adjoint_bytes(const Ctx &c, long npts_total, int gp_bytes)
{
    AdjWork w;
    return adjoint_carve(c, npts_total, gp_bytes, nullptr, &w);
}

void adjoint_reverse(const Ctx &c, const AdjWork &w, const RotorDev *rot, const BodyDev *bodies, int nbodies,
                     const int *ibm_iters, double power_seed, double dt, double t_np1)
{
    // the compute type of the local reverse maps is the storage type of the
    // tape's Gauss-point inputs
    auto spatial = w.gp_bytes == 4 ? spatial_adjoint<float> : spatial_adjoint<double>;
    const dim3 blk(32, 8), gcell((c.n[0] + 31) / 32, (c.n[1] + 7) / 8, c.n[2]);
    const size_t bytes4 = sizeof(double) * 4 * c.np;
    // IBM reverse (bodies act after the rotors, in the order added): lamP
    // goes from the state after the step to the state after the rotors
    for (int k = nbodies - 1; k >= 0; --k) {
        BodyDev b = bodies[k];
        b.niter = ibm_iters[k];
        ibm_adj_kernel<<<(int)((b.nbox + 255) / 256), 256, 0, c.stream>>>(w.lamP, c.np, c.P[0], c.P[1], b);
    }
    // ALM reverse: lamP holds lambda'' (state after the step) and becomes
    // lambda' (state before the forcing); per-point scale gradients in pts
    if (rot) {
        AlmAdjArgs A;
        for (int d = 0; d < 3; ++d) {
            A.P[d] = c.P[d];
            A.n[d] = c.n[d];
            A.x0[d] = c.x0[d];
            A.h[d] = c.hu[d];
        }
        A.np = c.np;
        A.Wp = w.Wp;
        A.lam = w.lamP;
        A.r = *rot;
        A.pts = w.pts;
        A.dt = dt;
        A.power_seed = power_seed;
        A.t = t_np1;
        const int npts = rot->nb * rot->np;
        alm_interp_adj_kernel<<<npts, 256, 0, c.stream>>>(A);
        alm_loads_adj_kernel<<<1, 256, 0, c.stream>>>(A);
        alm_sample_adj_kernel<<<(npts + 255) / 256, 256, 0, c.stream>>>(A, w.ptc, (long *)w.ptl);
        if (8 * npts <= kSampleSort)
            alm_sample_add_kernel<<<1, 1024, 0, c.stream>>>(A, w.ptc, (const long *)w.ptl);
        else
            alm_sample_add_serial_kernel<<<1, 1, 0, c.stream>>>(A, w.ptc, (const long *)w.ptl);
    }
    // stage 2: W' = P + dt^2/3 Lt(W*)
    rev_update_kernel<<<gcell, blk, 0, c.stream>>>(2, nullptr, w.lamP, nullptr, nullptr, w.lamLt, dt, c.np,
                                                   c.n[0], c.n[1], c.P[0], c.P[1]);
    cudaMemsetAsync(w.lamA, 0, bytes4, c.stream);
    if (w.A0f)
        spatial_adjoint_fused32(c, w, w.Wsf, nullptr, w.lamLt);
    else
        spatial(c, w, w.Ws, w.gps[1], nullptr, w.lamLt);
    ghost_adjoint(c, w, w.Ws);
    // stage 1: lamA (interior) is lambda of W*
    rev_update_kernel<<<gcell, blk, 0, c.stream>>>(1, w.lamA, w.lamP, w.lamW, w.lamL, w.lamLt, dt, c.np, c.n[0],
                                                   c.n[1], c.P[0], c.P[1]);
    cudaMemsetAsync(w.lamA, 0, bytes4, c.stream);
    if (w.A0f)
        spatial_adjoint_fused32(c, w, w.A0f, w.lamL, w.lamLt);
    else
        spatial(c, w, w.A0, w.gps[0], w.lamL, w.lamLt);
    ghost_adjoint(c, w, w.A0);
    add_interior_kernel<<<gcell, blk, 0, c.stream>>>(w.lamW, w.lamA, c.np, c.n[0], c.n[1], c.P[0], c.P[1]);
}

int bounds_flag_adjoint() { return bounds_flag_take(); }

}  // namespace gks
