// gks_internal.h -- declarations shared by the translation units of libgks.so
// (host context, device-resident scalars, kernel launchers). Not installed.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "gks_api.h"

namespace gks {

constexpr int G = 3;              // ghost layers (WENO5 needs 3)
constexpr int kMaxPartials = 1024;

enum : int { FLAG_NONFINITE = 1, FLAG_CFL = 2, FLAG_RANGE = 4, FLAG_TIMEOUT = 8 };

// Kernel groups for the optional per-launch event timing (gks_profile_*).
enum : int {
    K_PREP = 0, K_GHOST, K_CFL, K_FACE_EQ, K_FACE_FLUX, K_FLUX_UPDATE, K_ALM, K_IBM, K_MISC, K_NGROUPS
};

// Scalars that live in device memory so that a step needs no host round trip.
struct Scalars {
    double t;                       // time at the start of the current step
    double dt;                      // time step of the current step
    double cfl_number;              // CFL number of the last step
    unsigned long long maxu2_bits;  // max |U|^2 over interior cells (bits of a double >= 0)
    int flags;                      // FLAG_* raised by kernels
    int pad0;
    unsigned long long resid_bits;  // IBM residual max (bits of a double >= 0)
    int ibm_converged;
    int ibm_iters;
    double reserve[8];
};

// Host-side description of every device buffer and constant of one grid.
struct Ctx {
    int prec;                 // GKS_FP64 or GKS_FP32C
    int fp64_ds = 0;          // FP64 grids: reconstruction and flux in double-single arithmetic
    int n[3], P[3];
    long np;                  // element stride between component arrays (>= P0 P1 P2)
    long ncell;               // interior cells
    int bc[3][2];
    double lambda, theta, csound, mu, rho_ref, off;  // off = rho_ref (FP32C) or 0 (FP64)
    double cfl, dt_fixed, hmin;
    double inflow[4];         // rho, u, v, w
    double fbody[3];
    double x0[3], hu[3];      // origin and width of uniform axes (forcing)
    int xoff = 0;             // a slab's first cell in the x lattice of its group's domain (forcing)
    int uniform[3];
    cudaStream_t stream;

    void *state;              // FP64: double[4][np]; FP32C: float hi[4][np], lo[4][np]
    void *wk0;                // reconstruction input of stage 1 (FP64: == state)
    void *wk1;                // W* (reconstruction input of stage 2), R[4][np]
    void *pbuf;               // P = W + dt L + dt^2/6 Lt (FP64 double[4][np]; FP32C hi/lo)
    void *fq;                 // face equilibrium state + normal slope, R[8][nfq]
    long nfq;
    int e1p[3];               // padded t1 extent of the face box per direction (multiple of 4)
    CUtensorMap tmap[3];      // TMA descriptors of the face box per direction
    CUtensorMap tmapT[3];     // FP32C: the same with 20-row boxes (32 x 16 face tiles)
    // Optional (FP64): per direction, the 64 Gauss-point inputs of every face
    // (16 g + k arrays of stride ngp; g Gauss point, k = Q0, normal slope, t1
    // slope, t2 slope x 4 components), written by the flux kernels as double
    // (gp_bytes 8) or float (gp_bytes 4).
    void *gp_dir[3] = {nullptr, nullptr, nullptr};
    long ngp = 0;
    int gp_bytes = 8;
    // Stage 2 of a step may prepare the next step (the FP32 input, max |U|^2
    // outside the forcing boxes, which are redone after the forcing).
    int prep_next = 0;
    int nprep_box = 0;
    int prep_box[8][3][2];
    void *ff[3];              // face-averaged F0 and F1 of x and y faces, R[8][nff] (none for z)
    long nff[3];
    void *ih[3];              // R: inverse cell widths, padded index i + 3
    void *ihf[3];             // R: inverse centre distance at faces, f = 0..n
    double *h64[3];           // double: cell widths, padded index i + 3
    double *partials;         // double[kMaxPartials * 8]
    Scalars *scal;            // device scalars
    double *staging;          // >= 4 * ncell doubles, aliases the face-flux buffers

    // optional launch hook: called before (begin = 1) and after (begin = 0)
    // every kernel launch with the kernel group
    void (*mark)(void *ctx, int group, int begin) = nullptr;
    void *mark_ctx = nullptr;
};

inline void mark(const Ctx &c, int group, int begin)
{
    if (c.mark) c.mark(c.mark_ctx, group, begin);
}

// Message returned by gks_last_error(NULL) on this thread (gks_api.cu).
void record_error(const char *msg);
// Streaming multiprocessors of the current device (looked up once).
int sm_count();

// Debug-bounds builds: the index-check flag of each translation unit with
// kernels, taken and cleared (always 0 in a plain build).
int bounds_flag_stencil();
int bounds_flag_forcing();
int bounds_flag_adjoint();

// Launchers of the stencil path (gks_stencil.cu).
void launch_prep(const Ctx &c);                        // max |U|^2 into scal; FP32C: state -> wk0
void launch_prep_box(const Ctx &c, const int box[3][2]);   // the same over the interior cells of a box
void launch_ghost(const Ctx &c, void *w);              // 3 ghost layers of w (working type)
void launch_stage(const Ctx &c, int stage);            // face kernels + update
void launch_cfl(const Ctx &c);                          // dt from max |U| (after launch_prep)
void launch_advance(const Ctx &c);                      // t += dt
void launch_scatter_state(const Ctx &c, const double *d_src);  // compact FP64 -> state
void launch_scatter_state_prep(const Ctx &c, const double *d_src);   // + the prep of the new state
void launch_gather_state(const Ctx &c, double *d_dst);         // state -> compact FP64
void launch_face_state32(const Ctx &c, int d, const float *w);
void launch_diagnostics(const Ctx &c, double *d_out5);
void launch_fill_rest(const Ctx &c);                            // rho = 1, momentum 0
void launch_raw_copy(const Ctx &c, void *compact, int to_compact);  // stored arrays <-> compact
// out[i] = a[i] (+ b[i] if b) (+ off0 for i < n0), FP32 -> FP64, i < n
void launch_widen(const Ctx &c, const float *a, const float *b, double *out, long n, long n0, double off0);
// Slab groups (x-slabs of one domain on one device): the G x-planes of the
// working array next to x side `side_src` of `src` (all y and z rows, ghost
// rows included) into the G ghost planes on side `side_dst` of `dst`; and the
// largest max |U|^2 of the group into every slab's scalars.
void launch_halo_copy(const Ctx &src, const void *w_src, int side_src, const Ctx &dst, void *w_dst, int side_dst);
void launch_group_max_u2(Scalars *const *scal, int n, cudaStream_t stream);

// Actuator line (gks_forcing.cu).
struct RotorDev {
    int nb, np, correction, tip;
    double tip_g[2];    // g1 of the tip factor: axial, tangential
    double hub[3], omega, az0, radius, eps, rho_inf, uref;
    double rmin, rmax;  // smallest and largest point radius
    double *r, *chord, *twist, *width, *scale;  // device arrays
    double *X;          // 3 nb np positions of the last step
    float *Xr;          // the same relative to the hub, FP32 (projection screen)
    double norm, ie2;   // 1 / (eps^3 pi^1.5) and 1 / eps^2 of the Gaussian kernel
    double *F;          // 4 nb np: F_x, F_th, alpha, phi
    double *et;         // 2 nb: -sin th_b, cos th_b
    double *out;        // thrust[nb], torque[nb], power, cp, ct
    int box[3][2];      // interior cell box swept by the 3 eps supports
    int shared = 0;     // a slab's share of a neighbouring slab's rotor: its point buffers are the
                        // owner's, the owner computes the loads, this grid only spreads them
};
void launch_alm_spread(const Ctx &c, const RotorDev &r);   // projection only (a shared rotor)
void launch_alm(const Ctx &c, const RotorDev &r);
void launch_alm_loads(const Ctx &c, const RotorDev &r);   // loads only, no projection

// Adjoint of one step (gks_adjoint.cu). Buffers of the adjoint workspace:
// the tape of one step (what the reverse reads of the forward step) and the
// scratch of the reverse.
constexpr unsigned char kTapeMagicByte = 0x5A;   // hdr[0] bytes of a recorded tape
constexpr int kTapeHeader = 32;                    // doubles of the tape header
constexpr int kTapeMaxBodies = kTapeHeader - 4;    // IBM iteration counts a tape records
struct AdjWork {
    // tape
    double *hdr;                                          // [0] magic, [1] t_n, [2] dt, [3] gp_bytes,
                                                          // [4 + k] IBM iterations of body k
    double *A0, *Ws, *Wp;                                 // ghost-filled W^n, ghost-filled W*, state before the forcing
    float *A0f = nullptr, *Wsf = nullptr;                 // FP32C: the FP32 working arrays of both stages as the
                                                          // forward read them (rho - off, ghost-filled)
    const Ctx *c32 = nullptr;                             // FP32C: the grid's own context (FP32 widths, offset)
    void *gps[2][3];                                      // Gauss-point inputs of the forward (64 nG each)
    int gp_bytes;                                         // their storage: 8 (FP64 reverse) or 4 (FP32 reverse)
    long nG;                                              // component stride of gps
    // scratch
    double *lamA, *lamW, *lamP, *lamL, *lamLt;            // 4 * np each (padded indexing)
    double *lamGa;                                        // Gauss-point adjoints of one direction (64 nG)
    double *lamR, *lamFQ, *lamC;                          // per row / face buffers (FP32 reverse: floats)
    double *Asplit;                                       // FP32 reverse: the working array as hi, lo floats
    long nR;                                              // component stride of lamR
    double *uinf_part;                                    // per inflow ghost contribution
    long nuinf;
    double *red;                                          // partial sums of uinf_part (kRedBlocks)
    float *part = nullptr;                                // FP32C: per-tile face-box adjoints of one direction
    double *pts;                                          // per actuator point scratch (8 per point)
    double *ptc, *ptl;                                    // sampling-adjoint corner values (32) and cells (8, as long)
    double *scal;                                         // [0] grad U_inf (device accumulator)
    Scalars *sc;                                          // private time, dt and flags of the reverse
    double *ih64[3], *ihf64[3];                           // FP64 inverse widths (FP32C grids)
};
// Offsets from base (0 to size them); each returns its bytes. The full
// workspace of gks_step_adjoint is a tape followed by a scratch.
size_t adjoint_tape_carve(const Ctx &c, int gp_bytes, void *base, AdjWork *w);
size_t adjoint_scratch_carve(const Ctx &c, long npts_total, void *base, AdjWork *w);
size_t adjoint_bytes(const Ctx &c, long npts_total, int gp_bytes);
size_t adjoint_carve(const Ctx &c, long npts_total, int gp_bytes, void *base, AdjWork *w);
// Runs the reverse of one step from its tape in w (A0, W* in w.Ws, Wp, the
// face boxes and Gauss-point inputs of both stages; the rotor loads
// recomputed from Wp); accumulates into the per-point scratch and w.scal[0].
struct BodyDev;
// The local reverse maps (flux, WENO5 pair, equilibrium, transposed
// tangential passes) run in FP32 when the tape's Gauss-point inputs are
// stored as float (w.gp_bytes 4), else in FP64; FP64 state adjoints and sums.
// ibm_iters[k]: the direct-forcing iterations body k ran in the step.
void adjoint_reverse(const Ctx &c, const AdjWork &w, const RotorDev *rot, const BodyDev *bodies, int nbodies,
                     const int *ibm_iters, double power_seed, double dt, double t_np1);

// Immersed body (gks_forcing.cu).
struct BodyDev {
    int n, niter;
    double eps, tol;
    double *xyz, *vel;  // device, 3n each
    double *dS;         // device, n
    int box[3][2];
    long nbox;
    double *Vbar, *vbar, *phi;  // per box cell (vbar: 3 per cell)
    double *fsum;               // 3 per box cell
    double *out;                // force[3], iters, residual, residual history[niter]
    // back-interpolation weights W_{ijk->p} (static): CSR over points, columns
    // are box-local cell indices in (k, j, i) order
    long *csr_off;              // n + 1
    int *csr_cell;              // nnz
    double *csr_w;              // nnz
    long nnz;
    double *Ubox;               // 3 per box cell: cell velocity of the residual
    float *csr_wf, *Uboxf;      // FP32 copies of csr_w and Ubox (FP32C grids)
};
void launch_body_csr_count(const Ctx &c, const BodyDev &b, long *d_counts);
void launch_body_csr_fill(const Ctx &c, const BodyDev &b);
int body_box(const Ctx &c, const double *xyz, int n, double eps, int box[3][2]);
void launch_body_precompute(const Ctx &c, const BodyDev &b);
void launch_ibm(const Ctx &c, const BodyDev &b);

}  // namespace gks
