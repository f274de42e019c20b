// gks_device.cuh -- device building blocks shared by the forward stencil
// (gks_stencil.cu) and its adjoint (gks_adjoint.cu): physical constants,
// WENO5-JS, the tangential Gauss-point stencils, the closed-form
// gas-kinetic flux, and the TMA / mbarrier helpers. Internal header.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gks_ds.cuh"
#include "gks_internal.h"

namespace gks {
namespace dev {

template <typename R>
struct Phys {
    R lambda, theta, mu, off, sqlam, kE;
};

template <typename R>
Phys<R> make_phys(const Ctx &c)
{
    Phys<R> p;
    p.lambda = (R)c.lambda;
    p.theta = (R)c.theta;
    p.mu = (R)c.mu;
    p.off = (R)c.off;
    p.sqlam = (R)sqrt(c.lambda);
    p.kE = (R)(1.0 / (2.0 * sqrt(3.14159265358979323846 * c.lambda)));
    return p;
}

// Division in the working type: IEEE division in FP64; the two-instruction
// approximate division (2 ulp) in FP32, whose error is far below the FP32
// rounding of the stencil itself.
__device__ __forceinline__ double wdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float wdiv(float a, float b) { return __fdividef(a, b); }

// |U|^2 of a cell for the CFL time step, with every operation rounded
// explicitly so that each kernel that forms it gets the same bits: FP32C from
// hi + lo in FP32, FP64 from the state. max_u2 keeps a NaN.
__device__ __forceinline__ float cell_u2f(const float h[4], const float l[4])
{
    const float r = __fadd_rn(h[0], l[0]), a = __fadd_rn(h[1], l[1]);
    const float b = __fadd_rn(h[2], l[2]), c = __fadd_rn(h[3], l[3]);
    const float m2 = __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
    return __fdiv_rn(m2, __fmul_rn(r, r));
}
__device__ __forceinline__ double cell_u2(const float h[4], const float l[4]) { return (double)cell_u2f(h, l); }
__device__ __forceinline__ double cell_u2(const double w[4])
{
    const double m2 = __dadd_rn(__dadd_rn(__dmul_rn(w[1], w[1]), __dmul_rn(w[2], w[2])), __dmul_rn(w[3], w[3]));
    return __ddiv_rn(m2, __dmul_rn(w[0], w[0]));
}
__device__ __forceinline__ double max_u2(double a, double b) { return (b > a || b != b) ? b : a; }
__device__ __forceinline__ float max_u2f(float a, float b) { return (b > a || b != b) ? b : a; }

// Block-wide max of v (blockDim.x * blockDim.y threads, a multiple of 32,
// at most 1024) folded into *bits (a non-negative double) by one atomicMax.
__device__ __forceinline__ void block_max_to(double v, unsigned long long *bits)
{
    __shared__ double red[32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nw = (blockDim.x * blockDim.y) >> 5;
    for (int o = 16; o > 0; o >>= 1) v = max_u2(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nw; ++w) v = max_u2(v, red[w]);
        atomicMax(bits, (unsigned long long)__double_as_longlong(v));
    }
}

// Direction d: normal axis d, tangential axes t1, t2.
__host__ __device__ inline int tan1(int d) { return d == 0 ? 1 : 0; }
__host__ __device__ inline int tan2(int d) { return d == 2 ? 1 : 2; }

// WENO5-JS (Sec. 2): eps_w = 1e-6, power 2, linear weights 1/10, 6/10, 3/10
// on the candidate stencils (a,b,c), (b,c,d), (c,d,e) for the right face of
// the centre cell c.
// Both face values of the centre cell of q[0..4] (cells -2..2) from one set
// of Jiang-Shu smoothness indicators: the value at the right face (+1/2) and,
// with the stencils mirrored, at the left face (-1/2). The mirrored
// indicators are the same numbers in reverse order, so they are computed
// once. With s_k = (eps + beta_k)^2 the weights d_k / s_k are scaled by
// 10 s0 s1 s2 (linear weights 1/10, 6/10, 3/10 -> 1, 6, 3) and the 1/6 of the
// candidate polynomials moves into the one division per face value.
template <typename R>
__device__ __forceinline__ void weno5_pair(const R q[5], R &right, R &left)
{
    const R c13 = R(13.0 / 12.0), qq = R(0.25);
    const R a = q[0], b = q[1], c = q[2], d = q[3], e = q[4];
    R t = a - R(2) * b + c, u = a - R(4) * b + R(3) * c;
    R s0 = R(1e-6) + (c13 * t * t + qq * u * u);
    t = b - R(2) * c + d; u = b - d;
    R s1 = R(1e-6) + (c13 * t * t + qq * u * u);
    t = c - R(2) * d + e; u = R(3) * c - R(4) * d + e;
    R s2 = R(1e-6) + (c13 * t * t + qq * u * u);
    s0 *= s0; s1 *= s1; s2 *= s2;
    const R w02 = R(6) * (s0 * s2), s01 = s0 * s1, s12 = s1 * s2;
    // right face: candidates 6 p_k on (a,b,c), (b,c,d), (c,d,e)
    {
        const R p0 = R(2) * a - R(7) * b + R(11) * c;
        const R p1 = -b + R(5) * c + R(2) * d;
        const R p2 = R(2) * c + R(5) * d - e;
        const R w2 = R(3) * s01;
        right = wdiv(s12 * p0 + w02 * p1 + w2 * p2, R(6) * (s12 + w02 + w2));
    }
    // left face: candidates on (e,d,c), (d,c,b), (c,b,a) with indicators s2, s1, s0
    {
        const R p0 = R(2) * e - R(7) * d + R(11) * c;
        const R p1 = -d + R(5) * c + R(2) * b;
        const R p2 = R(2) * c + R(5) * b - a;
        const R w2 = R(3) * s12;
        left = wdiv(s01 * p0 + w02 * p1 + w2 * p2, R(6) * (s01 + w02 + w2));
    }
}

// erf(z), exp(-z^2) - 1 and exp(-z^2) of the half-space moments, z =
// sqrt(lambda) U. For |z| <= 1/2 (|U| up to 7 U_ref at Ma 0.1) the Maclaurin
// series
//   erf z = (2/sqrt pi) sum_n (-1)^n z^(2n+1) / (n! (2n+1)),
//   expm1 x = sum_n x^n / n!,
// FP32: n = 0..6 and 1..7 (first dropped terms below 4e-10 and 2e-9
// relative; within 2e-7 of the exact values after rounding); FP64: n = 0..12
// and 1..13 (dropped terms below 1e-17; within 3e-16 of libm); exp = 1 +
// expm1. Beyond 1/2 the library functions.
__device__ __forceinline__ void half_space_terms(double z, double &e, double &m1, double &ex)
{
    const double t = z * z, x = -t;
    if (fabs(z) <= 0.5) {
        constexpr double k = 1.1283791670955126;   // 2 / sqrt(pi)
        // c_n = k (-1)^n / (n! (2n+1))
        double p = k / (479001600.0 * 25.0);
        p = fma(p, t, -k / (39916800.0 * 23.0));
        p = fma(p, t, k / (3628800.0 * 21.0));
        p = fma(p, t, -k / (362880.0 * 19.0));
        p = fma(p, t, k / (40320.0 * 17.0));
        p = fma(p, t, -k / (5040.0 * 15.0));
        p = fma(p, t, k / (720.0 * 13.0));
        p = fma(p, t, -k / (120.0 * 11.0));
        p = fma(p, t, k / (24.0 * 9.0));
        p = fma(p, t, -k / (6.0 * 7.0));
        p = fma(p, t, k / (2.0 * 5.0));
        p = fma(p, t, -k / 3.0);
        p = fma(p, t, k);
        e = p * z;
        double q = 1.0 / 6227020800.0;   // 1/13!
        q = fma(q, x, 1.0 / 479001600.0);
        q = fma(q, x, 1.0 / 39916800.0);
        q = fma(q, x, 1.0 / 3628800.0);
        q = fma(q, x, 1.0 / 362880.0);
        q = fma(q, x, 1.0 / 40320.0);
        q = fma(q, x, 1.0 / 5040.0);
        q = fma(q, x, 1.0 / 720.0);
        q = fma(q, x, 1.0 / 120.0);
        q = fma(q, x, 1.0 / 24.0);
        q = fma(q, x, 1.0 / 6.0);
        q = fma(q, x, 0.5);
        q = fma(q, x, 1.0);
        m1 = q * x;
        ex = 1.0 + m1;
    } else {
        e = erf(z);
        m1 = expm1(x);
        ex = exp(x);
    }
}
__device__ __forceinline__ void half_space_terms(float z, float &e, float &m1, float &ex)
{
    const float t = z * z, x = -t;
    if (fabsf(z) <= 0.5f) {
        constexpr double k = 1.1283791670955126;   // 2 / sqrt(pi)
        float p = float(k / (720.0 * 13.0));
        p = fmaf(p, t, float(-k / (120.0 * 11.0)));
        p = fmaf(p, t, float(k / (24.0 * 9.0)));
        p = fmaf(p, t, float(-k / (6.0 * 7.0)));
        p = fmaf(p, t, float(k / (2.0 * 5.0)));
        p = fmaf(p, t, float(-k / 3.0));
        p = fmaf(p, t, float(k));
        e = p * z;
        float q = float(1.0 / 5040.0);
        q = fmaf(q, x, float(1.0 / 720.0));
        q = fmaf(q, x, float(1.0 / 120.0));
        q = fmaf(q, x, float(1.0 / 24.0));
        q = fmaf(q, x, float(1.0 / 6.0));
        q = fmaf(q, x, 0.5f);
        q = fmaf(q, x, 1.0f);
        m1 = q * x;
        ex = 1.0f + m1;
    } else {
        e = erff(z);
        m1 = expm1f(x);
        ex = expf(x);
    }
}

// Value conversion between a storage type and a compute type (identity, or
// double <-> double-single).
template <typename T>
__device__ __forceinline__ T cvt(double x) { return (T)x; }
template <>
__device__ __forceinline__ dsf cvt<dsf>(double x) { return to_ds(x); }
template <typename T>
__device__ __forceinline__ T cvt(float x) { return (T)x; }
template <typename T>
__device__ __forceinline__ T cvt(dsf x) { return (T)to_double(x); }
template <>
__device__ __forceinline__ dsf cvt<dsf>(dsf x) { return x; }

// Double-single: the same Maclaurin series as the FP64 version (n = 0..12
// and 1..13, dropped terms below 1e-17) in double-single arithmetic for
// |z| <= 1/2; beyond, the FP64 library functions.
__device__ __forceinline__ void half_space_terms(dsf z, dsf &e, dsf &m1, dsf &ex)
{
    if (fabsf(z.hi) <= 0.5f) {
        const dsf t = z * z, x = -t;
        constexpr double k = 1.1283791670955126;   // 2 / sqrt(pi)
        dsf p = dsf(k / (479001600.0 * 25.0));
        p = fma(p, t, dsf(-k / (39916800.0 * 23.0)));
        p = fma(p, t, dsf(k / (3628800.0 * 21.0)));
        p = fma(p, t, dsf(-k / (362880.0 * 19.0)));
        p = fma(p, t, dsf(k / (40320.0 * 17.0)));
        p = fma(p, t, dsf(-k / (5040.0 * 15.0)));
        p = fma(p, t, dsf(k / (720.0 * 13.0)));
        p = fma(p, t, dsf(-k / (120.0 * 11.0)));
        p = fma(p, t, dsf(k / (24.0 * 9.0)));
        p = fma(p, t, dsf(-k / (6.0 * 7.0)));
        p = fma(p, t, dsf(k / (2.0 * 5.0)));
        p = fma(p, t, dsf(-k / 3.0));
        p = fma(p, t, dsf(k));
        e = p * z;
        dsf q = dsf(1.0 / 6227020800.0);   // 1/13!
        q = fma(q, x, dsf(1.0 / 479001600.0));
        q = fma(q, x, dsf(1.0 / 39916800.0));
        q = fma(q, x, dsf(1.0 / 3628800.0));
        q = fma(q, x, dsf(1.0 / 362880.0));
        q = fma(q, x, dsf(1.0 / 40320.0));
        q = fma(q, x, dsf(1.0 / 5040.0));
        q = fma(q, x, dsf(1.0 / 720.0));
        q = fma(q, x, dsf(1.0 / 120.0));
        q = fma(q, x, dsf(1.0 / 24.0));
        q = fma(q, x, dsf(1.0 / 6.0));
        q = fma(q, x, dsf(0.5));
        q = fma(q, x, dsf(1.0));
        m1 = q * x;
        ex = dsf(1.0) + m1;
    } else {
        double de, dm, dx;
        half_space_terms(to_double(z), de, dm, dx);
        e = to_ds(de);
        m1 = to_ds(dm);
        ex = to_ds(dx);
    }
}

// Equilibrium state at a face (local frame, rho written as rho - off): the
// u>0 half of the left Maxwellian plus the u<0 half of the right one.
template <typename R>
__device__ __forceinline__ void face_equilibrium(const Phys<R> &ph, const R Ql[4], const R Qr[4], R Q0[4])
{
    const R rl = ph.off + Ql[0], rr = ph.off + Qr[0];
    const R Ul = wdiv(Ql[1], rl), Ur = wdiv(Qr[1], rr);
    R el, er, ml, mr, xl, xr;
    half_space_terms(ph.sqlam * Ul, el, ml, xl);
    half_space_terms(ph.sqlam * Ur, er, mr, xr);
    const R Pl = R(0.5) + R(0.5) * el;   // <u^0>_{u>0} of the left state
    const R Pr = R(0.5) - R(0.5) * er;   // <u^0>_{u<0} of the right state
    const R El = ph.kE * xl, Er = ph.kE * xr;
    Q0[0] = Ql[0] * Pl + Qr[0] * Pr + ph.off * (R(0.5) * (el - er));
    Q0[1] = Ql[1] * Pl + Qr[1] * Pr + (Ql[0] * El - Qr[0] * Er) + ph.off * (ph.kE * (ml - mr));
    Q0[2] = Ql[2] * Pl + Qr[2] * Pr;
    Q0[3] = Ql[3] * Pl + Qr[3] * Pr;
}

// Quartic through 5 face averages q[-2..2], at the Gauss points -g, +g of
// the centre cell, g = 1/(2 sqrt 3) (index space):
//   value(+-g) = E +- O, derivative(+-g) = Do +- De with s_k = q_k + q_-k,
//   a_k = q_k - q_-k and
//   E  = q0 + (s1 - 2 q0)/1080 - (s2 - 2 q0)/4320,
//   O  = (25 sqrt3 / 216) a1 - (7 sqrt3 / 432) a2,
//   Do = (2/3) a1 - (1/12) a2,
//   De = (13 sqrt3 / 54)(s1 - 2 q0) - (sqrt3 / 54)(s2 - 2 q0).
template <typename R>
__device__ __forceinline__ void tan_val(R qm2, R qm1, R q0, R qp1, R qp2, R &vm, R &vp)
{
    const R d1 = qp1 + qm1 - R(2) * q0, d2 = qp2 + qm2 - R(2) * q0;
    const R a1 = qp1 - qm1, a2 = qp2 - qm2;
    const R E = fma(d1, R(1.0 / 1080.0), fma(d2, R(-1.0 / 4320.0), q0));
    const R O = R(0.20046884346862007) * a1 - R(0.028065638085606807) * a2;
    vm = E - O;
    vp = E + O;
}

// The same values as tan_val as two 5-weight dot products (all on the FMA
// pipe). Used for rows that vanish identically in a uniform state (normal
// slopes, tangential derivatives), where the weights not summing exactly to
// one in floating point is harmless.
template <typename R>
__device__ __forceinline__ void tan_val_direct(R qm2, R qm1, R q0, R qp1, R qp2, R &vm, R &vp)
{
    const R w0 = R(-1.0 / 4320.0 + 0.028065638085606807), w1 = R(1.0 / 1080.0 - 0.20046884346862007);
    const R w2 = R(719.0 / 720.0);
    const R w3 = R(1.0 / 1080.0 + 0.20046884346862007), w4 = R(-1.0 / 4320.0 - 0.028065638085606807);
    vp = fma(w4, qp2, fma(w3, qp1, fma(w2, q0, fma(w1, qm1, w0 * qm2))));
    vm = fma(w0, qp2, fma(w1, qp1, fma(w2, q0, fma(w3, qm1, w4 * qm2))));
}

template <typename R>
__device__ __forceinline__ void tan_val_der(R qm2, R qm1, R q0, R qp1, R qp2, R &vm, R &vp, R &dm,
                                            R &dp)
{
    const R d1 = qp1 + qm1 - R(2) * q0, d2 = qp2 + qm2 - R(2) * q0;
    const R a1 = qp1 - qm1, a2 = qp2 - qm2;
    const R E = fma(d1, R(1.0 / 1080.0), fma(d2, R(-1.0 / 4320.0), q0));
    const R O = R(0.20046884346862007) * a1 - R(0.028065638085606807) * a2;
    const R Do = R(2.0 / 3.0) * a1 - R(1.0 / 12.0) * a2;
    const R De = R(0.41697519441472974) * d1 - R(0.032075014954979206) * d2;
    vm = E - O;
    vp = E + O;
    dm = Do - De;
    dp = Do + De;
}

// Gas-kinetic flux at one Gauss point (local frame: index 0 normal, 1 and 2
// tangential). The moments of f = g0 (1 - tau (a1 u + a2 v + a3 w + A) + A t)
// with the coefficients solved from the slopes and compatibility (Appendix)
// reduce to the closed form below (Chapman-Enskog structure, tau p = mu):
//   a.u + A = (1/theta) d_i U_j (c_i c_j - theta delta_ij),   c = u - U,
//   A = A0 + A_j c_j, A0 = -U.grad ln rho - div U,
//   A_k = -d_k ln rho - 2 lambda U_i d_i U_k,
//   F0 = (m_n, m_n U_k + p' delta_nk - mu (d_n U_k + d_k U_n)),
//   F1 = rho (A0 U_n + theta A_n, A0 (U_n U_k + theta delta_nk) + theta (A_k U_n + A_n U_k)),
// with p' = theta (rho - off): the constant theta off cancels in L.
// D1 and D2 are index-space tangential slopes; ih1, ih2 turn them into
// physical ones.
template <typename R, bool NEED_F0>
__device__ __forceinline__ void gk_flux(const Phys<R> &ph, const R q[4], const R Dn[4], const R D1[4],
                                        const R D2[4], R ih1, R ih2, R F0[4], R F1[4])
{
    const R rho = ph.off + q[0];
    const R inv = wdiv(R(1), rho);
    const R inv1 = inv * ih1, inv2 = inv * ih2;
    const R U0 = q[1] * inv, U1 = q[2] * inv, U2 = q[3] * inv;
    const R g0 = Dn[0] * inv, g1 = D1[0] * inv1, g2 = D2[0] * inv2;
    const R G00 = (Dn[1] - U0 * Dn[0]) * inv, G01 = (Dn[2] - U1 * Dn[0]) * inv,
            G02 = (Dn[3] - U2 * Dn[0]) * inv;
    const R G10 = (D1[1] - U0 * D1[0]) * inv1, G11 = (D1[2] - U1 * D1[0]) * inv1,
            G12 = (D1[3] - U2 * D1[0]) * inv1;
    const R G20 = (D2[1] - U0 * D2[0]) * inv2, G21 = (D2[2] - U1 * D2[0]) * inv2,
            G22 = (D2[3] - U2 * D2[0]) * inv2;
    const R th = ph.theta, tl = R(2) * ph.lambda;
    const R A0 = -(U0 * g0 + U1 * g1 + U2 * g2) - (G00 + G11 + G22);
    const R An = -g0 - tl * (U0 * G00 + U1 * G10 + U2 * G20);
    const R A1 = -g1 - tl * (U0 * G01 + U1 * G11 + U2 * G21);
    const R A2 = -g2 - tl * (U0 * G02 + U1 * G12 + U2 * G22);
    if (NEED_F0) {
        F0[0] = q[1];
        F0[1] = q[1] * U0 + th * q[0] - ph.mu * (G00 + G00);
        F0[2] = q[1] * U1 - ph.mu * (G01 + G10);
        F0[3] = q[1] * U2 - ph.mu * (G02 + G20);
    }
    F1[0] = rho * (A0 * U0 + th * An);
    F1[1] = rho * (A0 * (U0 * U0 + th) + th * (An * U0 + An * U0));
    F1[2] = rho * (A0 * (U0 * U1) + th * (A1 * U0 + An * U1));
    F1[3] = rho * (A0 * (U0 * U2) + th * (A2 * U0 + An * U2));
}

// ---- Packed FP32 pairs ----
//
// Two independent FP32 values that go through the same arithmetic (the two
// t1 Gauss points of a face) as one float2: the FP32x2 add, multiply and
// fused multiply-add of sm_100 and later do both in one instruction, which
// halves the issue slots of the arithmetic (the FP32 kernels are bound by
// instruction issue, not by the FMA pipe). Every operation is rounded
// explicitly, each lane exactly as its scalar counterpart (__fadd_rn,
// __fmul_rn, __fmaf_rn); nothing is contracted implicitly.
struct f2 {
    float2 v;
    f2() = default;
    __device__ __forceinline__ f2(float2 a) : v(a) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit f2(float a) : v(make_float2(a, a)) {}   // both lanes
    __device__ __forceinline__ explicit f2(double a) : f2((float)a) {}
};
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
// a - b as a + (-1) b: the product is exact, so one rounding as in __fsub_rn
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return fma(b, f2(-1.0f), a); }
__device__ __forceinline__ f2 &operator+=(f2 &a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2 &operator-=(f2 &a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2 operator-(f2 a) { return a * f2(-1.0f); }
// IEEE division per lane (the scalar FP32 path's a / b)
__device__ __forceinline__ f2 operator/(f2 a, f2 b) { return f2(__fdiv_rn(a.v.x, b.v.x), __fdiv_rn(a.v.y, b.v.y)); }
// the two-instruction approximate division of the scalar FP32 path, per lane
__device__ __forceinline__ f2 wdiv(f2 a, f2 b) { return f2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y)); }

// Two double-single values side by side (hi and lo parts as packed pairs):
// every operation is lane by lane the double-single operation of gks_ds.cuh
// (the same FP32 operations in the same order, so the same bits), with one
// packed instruction doing both lanes. Used for the flux of double-single
// grids at two Gauss points at once.
struct dsf2 {
    f2 hi, lo;
    dsf2() = default;
    __device__ __forceinline__ dsf2(f2 h, f2 l) : hi(h), lo(l) {}
    __device__ __forceinline__ dsf2(dsf a, dsf b) : hi(a.hi, b.hi), lo(a.lo, b.lo) {}
    __device__ __forceinline__ explicit dsf2(dsf a) : hi(a.hi), lo(a.lo) {}           // both lanes
    __device__ __forceinline__ explicit dsf2(double x) : dsf2(dsf(x)) {}
    __device__ __forceinline__ explicit dsf2(int x) : dsf2(dsf(x)) {}
    __device__ __forceinline__ dsf lane(int k) const
    {
        return k == 0 ? dsf(hi.v.x, lo.v.x) : dsf(hi.v.y, lo.v.y);
    }
};
__device__ __forceinline__ dsf2 two_sum(f2 a, f2 b)
{
    const f2 s = a + b;
    const f2 bb = s - a;
    return dsf2(s, (a - (s - bb)) + (b - bb));
}
// two_sum(a, -b): the same bits, with the negations folded into exact
// subtractions
__device__ __forceinline__ dsf2 two_diff(f2 a, f2 b)
{
    const f2 s = a - b;
    const f2 bb = s - a;
    return dsf2(s, (a - (s - bb)) - (b + bb));
}
__device__ __forceinline__ dsf2 fast_two_sum(f2 a, f2 b)
{
    const f2 s = a + b;
    return dsf2(s, b - (s - a));
}
__device__ __forceinline__ dsf2 operator+(dsf2 a, dsf2 b)
{
    dsf2 s = two_sum(a.hi, b.hi);
    const dsf2 t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ dsf2 operator-(dsf2 a, dsf2 b)
{
    dsf2 s = two_diff(a.hi, b.hi);
    const dsf2 t = two_diff(a.lo, b.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ dsf2 operator-(dsf2 a) { return dsf2(a.hi * f2(-1.0f), a.lo * f2(-1.0f)); }
__device__ __forceinline__ dsf2 operator*(dsf2 a, dsf2 b)
{
    const f2 p = a.hi * b.hi;
    f2 e = fma(a.hi, b.hi, p * f2(-1.0f));
    e = fma(a.hi, b.lo, e);
    e = fma(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ dsf2 operator/(dsf2 a, dsf2 b)
{
    const f2 q1(__fdiv_rn(a.hi.v.x, b.hi.v.x), __fdiv_rn(a.hi.v.y, b.hi.v.y));
    const dsf2 r = a - b * dsf2(q1, f2(0.0f));
    const f2 q2(__fdiv_rn(r.hi.v.x, b.hi.v.x), __fdiv_rn(r.hi.v.y, b.hi.v.y));
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ dsf2 &operator+=(dsf2 &a, dsf2 b) { return a = a + b; }
__device__ __forceinline__ dsf2 wdiv(dsf2 a, dsf2 b) { return a / b; }

__device__ __forceinline__ dsf2 &operator*=(dsf2 &a, dsf2 b) { return a = a * b; }
__device__ __forceinline__ dsf2 fma(dsf2 a, dsf2 b, dsf2 c) { return a * b + c; }

// half_space_terms of two double-single arguments: the series of both lanes
// as pairs when both lie in |z| <= 1/2, else lane by lane (the same bits as
// the scalar double-single version either way).
__device__ __forceinline__ void half_space_terms(dsf2 z, dsf2 &e, dsf2 &m1, dsf2 &ex)
{
    if (fabsf(z.hi.v.x) <= 0.5f && fabsf(z.hi.v.y) <= 0.5f) {
        const dsf2 t = z * z, x = -t;
        constexpr double k = 1.1283791670955126;   // 2 / sqrt(pi)
        dsf2 p = dsf2(k / (479001600.0 * 25.0));
        p = fma(p, t, dsf2(-k / (39916800.0 * 23.0)));
        p = fma(p, t, dsf2(k / (3628800.0 * 21.0)));
        p = fma(p, t, dsf2(-k / (362880.0 * 19.0)));
        p = fma(p, t, dsf2(k / (40320.0 * 17.0)));
        p = fma(p, t, dsf2(-k / (5040.0 * 15.0)));
        p = fma(p, t, dsf2(k / (720.0 * 13.0)));
        p = fma(p, t, dsf2(-k / (120.0 * 11.0)));
        p = fma(p, t, dsf2(k / (24.0 * 9.0)));
        p = fma(p, t, dsf2(-k / (6.0 * 7.0)));
        p = fma(p, t, dsf2(k / (2.0 * 5.0)));
        p = fma(p, t, dsf2(-k / 3.0));
        p = fma(p, t, dsf2(k));
        e = p * z;
        dsf2 q = dsf2(1.0 / 6227020800.0);   // 1/13!
        q = fma(q, x, dsf2(1.0 / 479001600.0));
        q = fma(q, x, dsf2(1.0 / 39916800.0));
        q = fma(q, x, dsf2(1.0 / 3628800.0));
        q = fma(q, x, dsf2(1.0 / 362880.0));
        q = fma(q, x, dsf2(1.0 / 40320.0));
        q = fma(q, x, dsf2(1.0 / 5040.0));
        q = fma(q, x, dsf2(1.0 / 720.0));
        q = fma(q, x, dsf2(1.0 / 120.0));
        q = fma(q, x, dsf2(1.0 / 24.0));
        q = fma(q, x, dsf2(1.0 / 6.0));
        q = fma(q, x, dsf2(0.5));
        q = fma(q, x, dsf2(1.0));
        m1 = q * x;
        ex = dsf2(1.0) + m1;
    } else {
        dsf e0, e1, m0, m1_, x0, x1;
        half_space_terms(z.lane(0), e0, m0, x0);
        half_space_terms(z.lane(1), e1, m1_, x1);
        e = dsf2(e0, e1);
        m1 = dsf2(m0, m1_);
        ex = dsf2(x0, x1);
    }
}

// face_equilibrium in double-single with the left and right half-space terms
// evaluated as one pair (the same bits as face_equilibrium<dsf>).
__device__ __forceinline__ void face_equilibrium_ds2(const Phys<dsf> &ph, const dsf Ql[4], const dsf Qr[4], dsf Q0[4])
{
    const dsf2 r = dsf2(ph.off) + dsf2(Ql[0], Qr[0]);
    const dsf2 U = wdiv(dsf2(Ql[1], Qr[1]), r);
    dsf2 e, m1, x;
    half_space_terms(dsf2(ph.sqlam) * U, e, m1, x);
    const dsf el = e.lane(0), er = e.lane(1), ml = m1.lane(0), mr = m1.lane(1);
    const dsf Pl = dsf(0.5) + dsf(0.5) * el;   // <u^0>_{u>0} of the left state
    const dsf Pr = dsf(0.5) - dsf(0.5) * er;   // <u^0>_{u<0} of the right state
    const dsf El = ph.kE * x.lane(0), Er = ph.kE * x.lane(1);
    Q0[0] = Ql[0] * Pl + Qr[0] * Pr + ph.off * (dsf(0.5) * (el - er));
    Q0[1] = Ql[1] * Pl + Qr[1] * Pr + (Ql[0] * El - Qr[0] * Er) + ph.off * (ph.kE * (ml - mr));
    Q0[2] = Ql[2] * Pl + Qr[2] * Pr;
    Q0[3] = Ql[3] * Pl + Qr[3] * Pr;
}

// ---- FP32 face state on packed pairs ----

// Approximate reciprocal per lane (the scalar FP32 path's __fdividef(1, x)).
__device__ __forceinline__ f2 wrcp(f2 x) { return f2(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y)); }

// weno5_pair of two components at once, every multiply-add fused explicitly
// and the constant factors folded into the candidates:
//  - the indicators are those of weno5_pair divided by 13/12 (the weights
//    depend on their ratios only): s_k = (eps 12/13 + t_k^2 + (3/13) u_k^2)^2,
//    with u_0 = t_0 + 2 (c - b) and u_2 = t_2 + 2 (c - d);
//  - the right-face weights times 10 s0 s1 s2 / 3 are s1 s2 / 3, 2 s0 s2 and
//    s0 s1 (mirrored for the left face), so with the candidates P_k = the
//    integer-coefficient ones divided by 18, 3 and 6 the face value is
//    (s12 P0 + s02 P1 + s01 P2) / (s12 / 3 + 2 s02 + s01).
__device__ __forceinline__ void weno5_pair2(const f2 q[5], f2 &right, f2 &left)
{
    const f2 m2(-2.0f), two(2.0f), eps(float(12e-6 / 13.0)), k(float(3.0 / 13.0));
    const f2 a = q[0], b = q[1], c = q[2], d = q[3], e = q[4];
    f2 t = fma(b, m2, a) + c, u = fma(c - b, two, t);
    f2 s0 = fma(t, t, fma(u * k, u, eps));
    t = fma(c, m2, b) + d;
    u = b - d;
    f2 s1 = fma(t, t, fma(u * k, u, eps));
    t = fma(d, m2, c) + e;
    u = fma(c - d, two, t);
    f2 s2 = fma(t, t, fma(u * k, u, eps));
    s0 = s0 * s0;
    s1 = s1 * s1;
    s2 = s2 * s2;
    const f2 s02 = s0 * s2, s01 = s0 * s1, s12 = s1 * s2;
    const f2 third(float(1.0 / 3.0));
    const f2 c3 = c * third, c53 = c * f2(float(5.0 / 3.0)), c1118 = c * f2(float(11.0 / 18.0));
    const f2 k19(float(1.0 / 9.0)), k718(float(-7.0 / 18.0)), k23(float(2.0 / 3.0)), km13(float(-1.0 / 3.0));
    const f2 k56(float(5.0 / 6.0)), km16(float(-1.0 / 6.0));
    {
        // right face: candidates on (a,b,c), (b,c,d), (c,d,e)
        const f2 P0 = fma(a, k19, fma(b, k718, c1118));
        const f2 P1 = fma(b, km13, fma(d, k23, c53));
        const f2 P2 = fma(e, km16, fma(d, k56, c3));
        right = fma(s12, P0, fma(s02, P1, s01 * P2)) * wrcp(fma(s12, third, fma(s02, two, s01)));
    }
    {
        // left face: the mirrored candidates with indicators s2, s1, s0
        const f2 P0 = fma(e, k19, fma(d, k718, c1118));
        const f2 P1 = fma(d, km13, fma(b, k23, c53));
        const f2 P2 = fma(a, km16, fma(b, k56, c3));
        left = fma(s01, P0, fma(s02, P1, s12 * P2)) * wrcp(fma(s01, third, fma(s02, two, s12)));
    }
}

// half_space_terms of two FP32 arguments: the series of both lanes as pairs
// when both lie in |z| <= 1/2 (the same operations per lane as the scalar
// series, so the same bits), else lane by lane.
__device__ __forceinline__ void half_space_terms(f2 z, f2 &e, f2 &m1, f2 &ex)
{
    if (fabsf(z.v.x) <= 0.5f && fabsf(z.v.y) <= 0.5f) {
        const f2 t = z * z, x = t * f2(-1.0f);
        constexpr double k = 1.1283791670955126;   // 2 / sqrt(pi)
        f2 p = f2(float(k / (720.0 * 13.0)));
        p = fma(p, t, f2(float(-k / (120.0 * 11.0))));
        p = fma(p, t, f2(float(k / (24.0 * 9.0))));
        p = fma(p, t, f2(float(-k / (6.0 * 7.0))));
        p = fma(p, t, f2(float(k / (2.0 * 5.0))));
        p = fma(p, t, f2(float(-k / 3.0)));
        p = fma(p, t, f2(float(k)));
        e = p * z;
        f2 q = f2(float(1.0 / 5040.0));
        q = fma(q, x, f2(float(1.0 / 720.0)));
        q = fma(q, x, f2(float(1.0 / 120.0)));
        q = fma(q, x, f2(float(1.0 / 24.0)));
        q = fma(q, x, f2(float(1.0 / 6.0)));
        q = fma(q, x, f2(0.5f));
        q = fma(q, x, f2(1.0f));
        m1 = q * x;
        ex = f2(1.0f) + m1;
    } else {
        half_space_terms(z.v.x, e.v.x, m1.v.x, ex.v.x);
        half_space_terms(z.v.y, e.v.y, m1.v.y, ex.v.y);
    }
}

// face_equilibrium with the components paired as (rho, m_n) and (m_t1, m_t2)
// (index 0 and 1 of L, R and Q0) and the half-space terms of the left and
// right states as one pair (lane 0 left, lane 1 right).
__device__ __forceinline__ void face_equilibrium2(const Phys<float> &ph, const f2 L[2], const f2 R[2], f2 Q0[2])
{
    const f2 r = f2(ph.off) + f2(L[0].v.x, R[0].v.x);
    const f2 U = f2(L[0].v.y, R[0].v.y) * wrcp(r);
    f2 e, m1, x;
    half_space_terms(f2(ph.sqlam) * U, e, m1, x);
    // (<u^0>_{u>0} of the left state, <u^0>_{u<0} of the right one)
    const f2 P = fma(e, f2(0.5f, -0.5f), f2(0.5f));
    const f2 E = f2(ph.kE) * x;
    const float d0 = (0.5f * ph.off) * (e.v.x - e.v.y);
    const float d1 = fmaf(L[0].v.x, E.v.x, -(R[0].v.x * E.v.y)) + (ph.kE * ph.off) * (m1.v.x - m1.v.y);
    const f2 Pl(P.v.x), Pr(P.v.y);
    Q0[0] = fma(R[0], Pr, fma(L[0], Pl, f2(d0, d1)));
    Q0[1] = fma(R[1], Pr, L[1] * Pl);
}

__device__ __forceinline__ Phys<dsf2> pair_phys(const Phys<dsf> &p)
{
    Phys<dsf2> q;
    q.lambda = dsf2(p.lambda);
    q.theta = dsf2(p.theta);
    q.mu = dsf2(p.mu);
    q.off = dsf2(p.off);
    q.sqlam = dsf2(p.sqlam);
    q.kE = dsf2(p.kE);
    return q;
}

// gk_flux at two Gauss points at once (the closed form above, every
// multiply-add fused explicitly). ph holds the FP32 constants.
template <bool NEED_F0>
__device__ __forceinline__ void gk_flux2(const Phys<float> &ph, const f2 q[4], const f2 Dn[4], const f2 D1[4],
                                         const f2 D2[4], f2 ih1, f2 ih2, f2 F0[4], f2 F1[4])
{
    const f2 m1(-1.0f);
    const f2 rho = f2(ph.off) + q[0];
    const f2 inv = wdiv(f2(1.0f), rho), ninv = inv * m1;
    const f2 inv1 = inv * ih1, inv2 = inv * ih2, ninv1 = ninv * ih1, ninv2 = ninv * ih2;
    const f2 U0 = q[1] * inv, U1 = q[2] * inv, U2 = q[3] * inv;
    // the logarithmic density slopes, negated: -d_k ln rho
    const f2 ng0 = Dn[0] * ninv, ng1 = D1[0] * ninv1, ng2 = D2[0] * ninv2;
    // G_ik = d_i U_k = (d_i m_k) / rho - U_k d_i ln rho
    const f2 G00 = fma(U0, ng0, Dn[1] * inv), G01 = fma(U1, ng0, Dn[2] * inv), G02 = fma(U2, ng0, Dn[3] * inv);
    const f2 G10 = fma(U0, ng1, D1[1] * inv1), G11 = fma(U1, ng1, D1[2] * inv1), G12 = fma(U2, ng1, D1[3] * inv1);
    const f2 G20 = fma(U0, ng2, D2[1] * inv2), G21 = fma(U1, ng2, D2[2] * inv2), G22 = fma(U2, ng2, D2[3] * inv2);
    const f2 th(ph.theta), ntl(-2.0f * ph.lambda);
    // A0 = -(U.g) - (G00 + G11 + G22); A_k = -g_k - 2 lambda U_i G_ik
    const f2 A0 = fma(U2, ng2, fma(U1, ng1, U0 * ng0)) - ((G00 + G11) + G22);
    const f2 An = fma(ntl, fma(U2, G20, fma(U1, G10, U0 * G00)), ng0);
    const f2 A1 = fma(ntl, fma(U2, G21, fma(U1, G11, U0 * G01)), ng1);
    const f2 A2 = fma(ntl, fma(U2, G22, fma(U1, G12, U0 * G02)), ng2);
    if (NEED_F0) {
        const f2 nmu(-ph.mu), n2mu(-2.0f * ph.mu);
        F0[0] = q[1];
        F0[1] = fma(q[1], U0, fma(th, q[0], G00 * n2mu));
        F0[2] = fma(q[1], U1, (G01 + G10) * nmu);
        F0[3] = fma(q[1], U2, (G02 + G20) * nmu);
    }
    F1[0] = rho * fma(A0, U0, th * An);
    F1[1] = rho * fma(A0, fma(U0, U0, th), f2(2.0f * ph.theta) * (An * U0));
    F1[2] = rho * fma(A0, U0 * U1, th * fma(A1, U0, An * U1));
    F1[3] = rho * fma(A0, U0 * U2, th * fma(A2, U0, An * U2));
}

constexpr int TX = 32, TY = 8;              // face tile
constexpr int SQ_W = TX + 4, SQ_H = TY + 4; // tile with the tangential halo
constexpr int SQ_N = 8 * SQ_H * SQ_W;
constexpr int ST_ROWS = SQ_H * TX;          // rows of the t1 pass
constexpr int ST_N = 24 * ST_ROWS;

// 8 consecutive values of a shared-memory row from a 16-byte aligned address,
// and 4 consecutive values to one.
__device__ __forceinline__ void lds8(const float *p, float q[8])
{
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
    q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
}
__device__ __forceinline__ void lds8(const double *p, double q[8])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double2 a = reinterpret_cast<const double2 *>(p)[i];
        q[2 * i] = a.x;
        q[2 * i + 1] = a.y;
    }
}
__device__ __forceinline__ void sts4(float *p, const float q[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(q[0], q[1], q[2], q[3]);
}
__device__ __forceinline__ void sts4(double *p, const double q[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(q[0], q[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(q[2], q[3]);
}
__device__ __forceinline__ void lds8(const dsf *p, dsf q[8])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 a = reinterpret_cast<const float4 *>(p)[i];
        q[2 * i] = dsf(a.x, a.y);
        q[2 * i + 1] = dsf(a.z, a.w);
    }
}
__device__ __forceinline__ void sts4(dsf *p, const dsf q[4])
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(q[0].hi, q[0].lo, q[1].hi, q[1].lo);
    reinterpret_cast<float4 *>(p)[1] = make_float4(q[2].hi, q[2].lo, q[3].hi, q[3].lo);
}

static_assert(TX * TY == 256 && SQ_H == 12 && TX == 32, "t1-pass task split assumes 32 x 8 tiles");

// Taller face tiles (FP32C x and y faces): 32 x 16 faces, each thread two
// faces adjacent along t2, so that the t2 pass reads 6 rows for 2 faces
// instead of 5 for 1 and the t1 pass recomputes 4 halo rows per 16 instead
// of per 8.
constexpr int TYT = 16;
constexpr int SQ_HT = TYT + 4;
constexpr int SQ_NT = 8 * SQ_HT * SQ_W;
constexpr int ST_ROWS_T = SQ_HT * TX;
constexpr int ST_NT = 24 * ST_ROWS_T;

// t1 pass of one tile of H rows (with the tangential halo): values and
// t1-derivatives of Q0, values of the normal slope, at the two t1 Gauss
// points, for every row of the tile. 64 H equal tasks (Q0 or slope,
// component, row, group of 4 columns), H / 4 per thread: a task reads 8
// consecutive values of its row and writes 4 columns; the lanes of a warp
// share the kind and the component (8 H is a multiple of 32).
template <typename R, typename C, int H = SQ_H>
__device__ __forceinline__ void tile_t1_pass(const R *sq, C *st, int tid)
{
    static_assert(H % 4 == 0, "a warp's tasks share kind and component");
    constexpr int NQ = 32 * H, NV = 8 * H, ROWS = H * TX;
#pragma unroll
    for (int j = 0; j < H / 4; ++j) {
        const int task = tid + j * 256;
        const int kind = task >= NQ, rem = task - kind * NQ, v = rem / NV, rc = rem - v * NV;
        const int r = rc >> 3, cg = rc & 7;
        C q[8];
        lds8(sq + ((kind * 4 + v) * H + r) * SQ_W + 4 * cg, q);
        C *o = st + r * TX + 4 * cg;
        if (kind == 0) {
            C vm[4], vp[4], dm[4], dp[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) tan_val_der(q[i], q[i + 1], q[i + 2], q[i + 3], q[i + 4], vm[i], vp[i], dm[i], dp[i]);
            sts4(o + (v * 4 + 0) * ROWS, vm);
            sts4(o + (v * 4 + 1) * ROWS, vp);
            sts4(o + (v * 4 + 2) * ROWS, dm);
            sts4(o + (v * 4 + 3) * ROWS, dp);
        } else {
            C vm[4], vp[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) tan_val_direct(q[i], q[i + 1], q[i + 2], q[i + 3], q[i + 4], vm[i], vp[i]);
            sts4(o + (16 + v * 2 + 0) * ROWS, vm);
            sts4(o + (16 + v * 2 + 1) * ROWS, vp);
        }
    }
}

template <typename R>
constexpr size_t flux_smem_bytes()
{
    return (size_t)(SQ_N + ST_N) * sizeof(R) + 2 * sizeof(unsigned long long);
}
constexpr size_t flux_tall_smem_bytes() { return (size_t)(SQ_NT + ST_NT) * sizeof(float) + 2 * sizeof(unsigned long long); }


// ---- TMA and mbarrier helpers (sm_90+ PTX) ----

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One bulk tensor copy of the (TX+4) x (TY+4) x 1 x 8 face box starting at
// (c0, c1, c2, 0) into dst; completion is signalled on bar with the byte
// count.
__device__ __forceinline__ void tma_load_tile(const CUtensorMap *map, void *dst, uint64_t *bar, int c0, int c1,
                                              int c2, uint32_t bytes)
{
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(0), "r"(b)
        : "memory");
}

// 4- or 8-byte asynchronous copy global -> shared (completion through
// cp.async groups), and the group fences.
__device__ __forceinline__ void cp_async(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)),
                 "l"((unsigned long long)__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async(double *dst, const double *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)),
                 "l"((unsigned long long)__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async(dsf *dst, const dsf *src)
{
    cp_async(reinterpret_cast<double *>(dst), reinterpret_cast<const double *>(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Wait for phase `parity` of bar; gives up after ~1 s of SM clock and
// returns false (the caller raises FLAG_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t b = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
}


}  // namespace dev
}  // namespace gks
