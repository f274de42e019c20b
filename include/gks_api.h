/*
 * gks_api.h -- C ABI of the GB300 (sm_103a) library libgks.so: one two-stage
 * fourth-order (S2O4) step of the high-order gas-kinetic scheme (GKS) for 3D
 * weakly compressible isothermal flow on a structured grid, with actuator-line
 * (ALM) and immersed-boundary (IBM) body forcing.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: GKS_OK (0) or a negative error
 *     code below. gks_last_error(g) returns a message for the last failure on
 *     a grid (a static string for calls without a grid).
 *   - Host arrays passed in are copied during the call; the library keeps no
 *     pointer to them.
 *   - Device memory for the state and the work space is owned by the caller
 *     (for example torch tensors): the library never frees it, and it must
 *     outlive the grid. The library owns only the small device buffers it
 *     allocates for actuator lines and immersed bodies (freed by
 *     gks_destroy_grid); a time step allocates nothing (with gks_set_graphs
 *     the first captured step also creates the graph and a capture stream,
 *     likewise freed by gks_destroy_grid).
 *   - Work is enqueued on the CUDA stream given in the grid description (NULL
 *     = the legacy default stream). Calls that return results to the host
 *     synchronise that stream.
 *   - Calls on one grid are not thread safe.
 *
 * Citations name the paper (Huo, Pan, Cao et al., "High-order gas-kinetic
 * scheme for numerical simulations of wind turbine with nacelle and tower
 * using ALM and IBM") by section, equation or appendix.
 */
#ifndef GKS_API_H
#define GKS_API_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GKS_OK 0
#define GKS_ERR_ARG (-1)       /* invalid argument or handle                        */
#define GKS_ERR_CUDA (-2)      /* a CUDA runtime call failed                        */
#define GKS_ERR_NONFINITE (-3) /* a non-finite value appeared in the updated state  */
#define GKS_ERR_CFL (-4)       /* fixed time step above the CFL limit given        */
#define GKS_ERR_STATE (-5)     /* call not allowed in the current state             */
#define GKS_ERR_RANGE (-6)     /* actuator point outside the sampled interior       */
#define GKS_ERR_DEBUG_BOUNDS (-7) /* debug-bounds build only: a kernel met an index
                                     outside its buffer (the access was skipped)     */

#define GKS_MAX_BLADES 8

/* Arithmetic of the step. GKS_FP64: everything in FP64. GKS_FP32C:
 * reconstruction and flux in FP32 on density perturbations rho - rho_ref,
 * the conserved state carried as compensated FP32 pairs (hi + lo) updated
 * with an error-free two-sum; global reductions and rotor loads summed in
 * FP64. */
typedef enum { GKS_FP64 = 0, GKS_FP32C = 1 } gks_precision;

/* Boundary kinds (Sec. 4): periodic; no-slip isothermal wall (mirror, all
 * momenta negated); slip / symmetry wall (mirror, normal momentum negated);
 * inflow with prescribed velocity and density from the outgoing isothermal
 * Riemann invariant U -/+ C ln rho; extrapolation (zero-gradient) outflow.
 * GKS_BC_EXCHANGE (x faces only): the side of an x-slab that borders the
 * next slab of a slab group; its ghost planes come from that slab
 * (gks_slab_step, Sec. 3's decomposition of the domain into x-slabs), never
 * from a boundary rule. */
typedef enum {
    GKS_BC_PERIODIC = 0,
    GKS_BC_NOSLIP = 1,
    GKS_BC_SLIP = 2,
    GKS_BC_INFLOW = 3,
    GKS_BC_OUTFLOW = 4,
    GKS_BC_EXCHANGE = 5
} gks_bc;

typedef struct gks_grid gks_grid;

/* Grid description (Sec. 2; Sec. 4 for the boundary kinds).
 *   n[d]       cells along axis d (x, y, z). >= 3 for non-periodic axes, >= 1
 *              for periodic ones (n = 1 collapses an axis); at most 2^24
 *              per axis and (n[0]+1)(n[1]+1)(n[2]+1) <= 2e9.
 *   faces[d]   host array of n[d]+1 strictly increasing face coordinates
 *              (uniform or stretched; reconstruction is done in index space
 *              and derivatives use the local cell widths).
 *   mach,u_ref lambda = mach^2 / (2 u_ref^2) of the isothermal Maxwellian
 *              (Sec. 2); sound speed C = sqrt(1 / (2 lambda)).
 *   mu         dynamic viscosity; collision time tau = mu / p, p = rho/(2 lambda).
 *   bc[d][s]   boundary kind at the low (s=0) and high (s=1) end of axis d;
 *              periodic must be set on both ends or neither.
 *   precision  gks_precision.
 *   cfl        CFL number of Sec. 2: dt = cfl min(dx,dy,dz) / (|U|max + C).
 *   dt_fixed   > 0: use this time step instead; cfl then is the largest CFL
 *              number allowed (GKS_ERR_CFL above it; cfl <= 0 disables).
 *   rho_ref    reference density of the FP32C perturbation form (> 0); not
 *              used by GKS_FP64.
 *   stream     cudaStream_t (as void*) on which every call enqueues work. */
typedef struct {
    int n[3];
    const double *faces[3];
    double mach, u_ref, mu;
    int bc[3][2];
    int precision;
    double cfl, dt_fixed;
    double rho_ref;
    void *stream;
} gks_grid_desc;

/* Bytes of device memory the caller must provide for the state and for the
 * work space of a grid with this description. Both buffers must be 256-byte
 * aligned. Returns GKS_ERR_ARG for an invalid description. */
int gks_workspace_bytes(const gks_grid_desc *desc, size_t *state_bytes, size_t *work_bytes);

/* Create a grid over caller-owned device buffers d_state and d_work of the
 * sizes returned by gks_workspace_bytes. The state is set to rest
 * (rho = 1, momentum 0), the time to 0. *out receives the handle. */
int gks_create_grid(const gks_grid_desc *desc, void *d_state, void *d_work, gks_grid **out);

/* Release the handle and the library-owned device buffers (not d_state or
 * d_work). Synchronises the grid's stream first. */
int gks_destroy_grid(gks_grid *g);

/* Message for the last failure on g (or for a failure without a grid). */
const char *gks_last_error(const gks_grid *g);

/* Change the stream used by subsequent calls. */
int gks_set_stream(gks_grid *g, void *stream);

/* Set / get the conserved state (rho, rho U, rho V, rho W) of the interior
 * cells from / to a host FP64 array of 4 * N values, component-major, x
 * fastest then y then z (N = n0 n1 n2). Page-locked host memory makes the
 * copy asynchronous for gks_set_state; gks_get_state synchronises. For
 * GKS_FP32C the value is split into hi = fl32(q), lo = fl32(q - hi). */
int gks_set_state(gks_grid *g, const double *h_state);
int gks_get_state(gks_grid *g, double *h_state);

/* Inflow state used by GKS_BC_INFLOW faces: density (the ghost density is
 * set from the Riemann invariant; this value is the reference of the
 * boundary) and the prescribed velocity. Sec. 4.3. */
int gks_set_inflow(gks_grid *g, double rho, double u, double v, double w);

/* Constant body force per unit volume added to the momentum after each S2O4
 * update (channel driving force of Sec. 4.1: rho U += dt f). */
int gks_set_body_force(gks_grid *g, double fx, double fy, double fz);

/* Actuator-line rotor (Sec. 3.1). The rotor axis is +x; blade b's azimuth at
 * time t is azimuth0 + omega t + 2 pi b / n_blades, its points sit at
 * hub + r (0, cos th, sin th) and move along e_th = (0, -sin th, cos th).
 * Per point (host arrays of n_pts, copied): radius r, chord, twist (rad) and
 * element width. Loads use the synthetic polar C_L = clip(2 pi sin a, +-1.4),
 * C_D = 0.01 + 0.02 a^2, L and D = 1/2 rho_inf c w C |U_rel|^2 (Eq.
 * (axial-tangential)), F_x = L cos phi + D sin phi, F_th = L sin phi -
 * D cos phi, and are projected with the Gaussian of Eq. (Gaussian) cut at
 * 3 eps. correction != 0 applies the free-stream velocity correction of
 * Sec. 3.1 once, with C_D of the uncorrected angle. radius and u_inf_ref
 * normalise C_P and C_T (Sec. 4.4.1). tip_correction != 0 multiplies F_x and
 * F_th by the tip factors of Eq. (tip-correction) (Sec. 4.4):
 *   f = (2/pi) acos(exp(-g1 N (R - r) / (2 r |sin phi|))),
 *   g1 = exp(-c1 (N lambda - c2)) + 0.1, lambda = omega R / u_inf_ref,
 * with (c1, c2) = (0.1219, 21.52) for F_x and (0.0984, 13.026) for F_th,
 * N = n_blades, R = radius; f = 0 for r >= R. All axes must be uniform. */
typedef struct {
    int n_blades, n_pts;
    double hub[3];
    double omega, azimuth0, radius, eps;
    double rho_inf, u_inf_ref;
    const double *r, *chord, *twist, *width;
    int correction;
    int tip_correction;
} gks_rotor_desc;

/* Add a rotor; *id receives its object id. Not allowed after the first step
 * (GKS_ERR_STATE). Allocates small library-owned device buffers. */
int gks_add_actuator_lines(gks_grid *g, const gks_rotor_desc *desc, int *id);

/* gks_set_slab_lattice: for a slab of a slab group (gks_slab_step), the
 * uniform x lattice of the group's whole domain, on which the forcing places
 * cell centres and actuator and IB points: its origin x0, cell width hx, and
 * the number of the domain's cells before this slab's first one. With it a
 * slab's forcing has the bits of the whole grid's. Call it before adding
 * rotors or bodies (GKS_ERR_STATE otherwise); the slab's x axis must be
 * uniform and its first face must lie on that lattice (GKS_ERR_ARG
 * otherwise). gks_slab_step requires it on every slab of a group that holds
 * rotors or bodies. */
int gks_set_slab_lattice(gks_grid *g, double x0, double hx, int cells_before);

/* gks_share_actuator_lines: in a slab group, give slab g its share of rotor id
 * of the neighbouring slab `owner` whose kernel support reaches their cut:
 * in every group step the owner samples the flow and computes the point
 * forces and loads, then g spreads those point forces into its own cells.
 * *id_out receives the share's object id on g; gks_forces on it reports the
 * owner's loads. g and owner must have the same precision and x lattice
 * (gks_set_slab_lattice) and g must not have been stepped (GKS_ERR_ARG,
 * GKS_ERR_STATE); GKS_ERR_RANGE if the support misses g. The share reads the
 * owner's point buffers (it allocates nothing): destroy the two together. A
 * grid holding a share steps only within its group (gks_step returns
 * GKS_ERR_STATE). The rotors' own exchange-side check happens in
 * gks_slab_step: a rotor whose support reaches a cut must be shared with the
 * slab behind the cut. */
int gks_share_actuator_lines(gks_grid *owner, int id, gks_grid *g, int *id_out);

/* Per-point force scales s (host array of n_blades * n_pts, blade-major)
 * multiplying every point force of rotor id; 1 by default. */
int gks_set_force_scales(gks_grid *g, int id, const double *h_scales);

/* Add a stationary or moving immersed body (Sec. 3.2) of n Lagrangian
 * points: xyz (3n host values, point-major), surface element areas dS (n),
 * point velocities vel (3n, or NULL for a stationary body; the points keep
 * their positions, so vel prescribes the surface velocity of a body whose
 * shape stays in place, e.g. one turning about its own axis), the kernel width
 * eps of the truncated Gaussian used both ways, the number of direct-forcing
 * iterations niter (>= 1) and a residual tolerance tol (0 = always niter
 * iterations). V_p = Delta dS with Delta = (dx dy dz)^(1/3). The cell fields
 * Vbar, vbar and phi = min(Vbar/|Omega|, 1) are computed once here. Kernel
 * supports are truncated to interior cells. All axes must be uniform. */
int gks_add_ib_points(gks_grid *g, int n, const double *xyz, const double *dS, const double *vel,
                      double eps, int niter, double tol, int *id);

/* Advance nsteps S2O4 steps (Sec. 2; forcing after each update, end of Sec. 3.2:
 * body force, rotors in the order added, then bodies in the order added).
 * Synchronises the stream at the end and reports GKS_ERR_NONFINITE,
 * GKS_ERR_CFL or GKS_ERR_RANGE raised on the device. t_out (may be NULL)
 * receives the time after the last step. */
int gks_step(gks_grid *g, int nsteps, double *t_out);

/* gks_slab_step: advance a slab group, nslab grids that split one domain
 * along x (the paper's multi-GPU decomposition, Sec. 3: x-slabs with a halo
 * exchange per stage), by nsteps steps, on one device. slabs[0 .. nslab-1]
 * are in the order of increasing x; each was created by gks_create_grid with
 * its own share of the x faces and GKS_BC_EXCHANGE on every x side that
 * borders another slab (slab s's high side and slab s+1's low side; slab 0's
 * low and slab nslab-1's high side for a periodic x axis, which the group
 * then closes). Per stage, after each slab's ghost fill, the three interior
 * x-planes of the working array next to each exchange side (all y and z
 * rows, ghost rows included) are copied into the neighbour's ghost planes;
 * the CFL time step takes the largest |U|^2 of all slabs and the smallest
 * cell width of all slabs; each slab applies its own rotors and bodies. A
 * rotor's kernel support may reach a cut if the slab behind the cut holds a
 * share of it (gks_share_actuator_lines; GKS_ERR_RANGE otherwise): owners
 * compute their rotors' loads and spread them, then the shares spread the
 * owners' point forces, then the bodies are applied. Bodies must stay inside
 * their slab (gks_add_ib_points returns GKS_ERR_RANGE otherwise). With
 * rotors or bodies, every slab needs the domain's x lattice
 * (gks_set_slab_lattice). The first call
 * also gives each exchange side's ghost cells the neighbour's cell widths
 * (the geometry tables a grid of the whole domain has at the cut), so the
 * state of every slab then has the bits that grid would have.
 * Requirements (GKS_ERR_ARG otherwise): 1 <= nslab <= 64; the same precision,
 * arithmetic, y and z cells, faces and boundary kinds, physics (Mach, U_ref,
 * mu, CFL or fixed dt, rho_ref) and stream on every slab; exchange sides
 * exactly where stated above; no CUDA graphs (gks_set_graphs) on a slab. Synchronises the stream at the end
 * and reports device flags like gks_step, per slab. t_out (may be NULL)
 * receives the time after the last step. Allocates nothing. */
int gks_slab_step(gks_grid *const *slabs, int nslab, int nsteps, double *t_out);
/* The same steps, enqueued on the grid's stream without synchronising:
 * device-side errors stay flagged on the device and are reported by the next
 * gks_step or gks_sync. */
int gks_step_async(gks_grid *g, int nsteps);
/* Synchronise the grid's stream, report errors flagged on the device as
 * gks_step does, and give the current time (t_out may be NULL). */
int gks_sync(gks_grid *g, double *t_out);
/* With on != 0, gks_step and gks_step_async replay a CUDA graph of one step
 * once the grid is in its steady state (a plain step done, the next step's
 * input prepared by the last one, at most 8 forcing objects, profiling
 * timing and NVTX off): one graph launch per step instead of one launch per
 * kernel, which pays on small grids whose steps are launch-bound. The graph
 * is captured when first needed and again after gks_set_inflow,
 * gks_set_body_force or gks_profile_enable; results are the same bits as
 * plain steps. Off by default. */
int gks_set_graphs(gks_grid *g, int on);

/* Arithmetic of the reconstruction and flux kernels of an FP64 grid:
 * double_single = 0 (default) runs them in FP64; 1 runs them in double-single
 * arithmetic (each value an unevaluated sum of two FP32 numbers, about 48
 * significant bits, error-free transformations of Knuth and Dekker) on the
 * FP32 pipe, with the state, the face buffers, the stage update and every
 * sum still in FP64 and the transcendental terms of the equilibrium state
 * evaluated in FP64. GB300 runs FP64 at about 1/64 of its FP32 rate, so the
 * double-single step is several times faster; its results agree with the
 * FP64 ones to about 1e-13 relative (not bit for bit). Recorded steps of the
 * adjoint (gks_step_record) always run in FP64. Applies from the next step.
 * Returns GKS_ERR_STATE for an FP32C grid. */
int gks_set_fp64_arithmetic(gks_grid *g, int double_single);

/* Current time and the last time step (synchronises). */
int gks_get_time(gks_grid *g, double *t, double *dt_last);
int gks_set_time(gks_grid *g, double t);

/* Loads of object id from the last step (synchronises).
 * Rotor: thrust and torque per blade, power = omega sum(torque),
 *   C_P = 2 omega T' / (rho pi R^2 U^3), C_T = 2 D' / (rho pi R^2 U^2)
 *   (Sec. 4.4.1), summed in FP64. h_points (may be NULL) receives 4 arrays of
 *   n_blades * n_pts: F_x, F_th, angle of attack, flow angle.
 * Body: the force on the structure (minus the summed cell forces of Eq.
 *   (force-ibm)), the iterations done and the last residual
 *   max_p |v_p - sum W U|. h_points (may be NULL) receives the residual of
 *   each iteration (niter values; zero where not evaluated). */
typedef struct {
    int kind; /* 0 rotor, 1 body */
    int n_blades;
    double thrust[GKS_MAX_BLADES], torque[GKS_MAX_BLADES];
    double power, cp, ct;
    double body_force[3];
    int iters;
    double residual;
} gks_forces_out;
int gks_forces(gks_grid *g, int id, gks_forces_out *out, double *h_points);

/* The load record of object id, copied on the grid's stream into h_out
 * without synchronising: asynchronous when h_out is page-locked; the caller
 * synchronises the stream (an event, a later call that synchronises) before
 * reading it. The record holds what gks_forces reports, as doubles:
 *   rotor: thrust[n_blades], torque[n_blades], power, C_P, C_T;
 *   body: force[3], iterations, residual, two internal words, then the
 *         residual of each iteration (niter values).
 * gks_forces_record_len gives its length in doubles; n is the room at h_out
 * (GKS_ERR_ARG if smaller). */
int gks_forces_record_len(const gks_grid *g, int id, size_t *n);
int gks_forces_async(gks_grid *g, int id, double *h_out, size_t n);

/* Mass, momentum (3) and kinetic energy summed over interior cells with
 * their volumes, in FP64 (synchronises). */
int gks_diagnostics(gks_grid *g, double out[5]);

/* Checkpoint: the interior state in its stored precision, the time and the
 * step count. gks_checkpoint_bytes gives the blob size. */
int gks_checkpoint_bytes(gks_grid *g, size_t *bytes);
int gks_save_state(gks_grid *g, void *h_blob, size_t bytes);
int gks_load_state(gks_grid *g, const void *h_blob, size_t bytes);

/* Layout of the caller-owned state buffer: out[0..2] padded extents (n + 6),
 * out[3] element bytes (8 for FP64, 4 for FP32C), out[4] number of arrays
 * (4 for FP64: rho, rho U, rho V, rho W; 8 for FP32C: the 4 hi arrays then
 * the 4 lo arrays), out[5] element stride between arrays, out[6] ghost width
 * (3). Interior cell (i,j,k) of array a is element
 * a*out[5] + (i+3) + out[0]*((j+3) + out[1]*(k+3)). */
int gks_state_layout(const gks_grid *g, long out[7]);

/* Device-side state exchange: the same compact FP64 layout as
 * gks_set_state / gks_get_state (4 * N values, component-major, x fastest),
 * in device memory. Asynchronous on the grid's stream. */
int gks_set_state_device(gks_grid *g, const double *d_state);
int gks_get_state_device(gks_grid *g, double *d_state);

/* Adjoint of one step (reverse mode): for a functional J of the state
 * after the step, given lambda^{n+1} = dJ/dW^{n+1}, computes
 * lambda^n = dJ/dW^n (through the ghost fill, both S2O4 stages with their
 * WENO5 reconstruction, equilibrium state, tangential Gauss-point
 * reconstruction and gas-kinetic flux (Sec. 2, Appendix), and the ALM
 * sampling, loads and Gaussian projection (Sec. 3.1)), and adds to
 * *h_grad_scales (n_blades * n_pts, rotor 0) the gradient with respect to
 * the per-point force scales and to *h_grad_uinf the gradient with respect
 * to the inflow speed u (the x velocity of gks_set_inflow), both through
 * this step only. power_seed is dJ/dP for the rotor power P of this step.
 *   d_adj_work  device workspace of gks_adjoint_workspace_bytes bytes
 *               (256-byte aligned, caller-owned);
 *   t_n         time at the start of the step;
 *   d_state_n   device, W^n (compact FP64 layout);
 *   d_adj_np1   device, lambda^{n+1} (compact FP64);
 *   d_adj_n     device, receives lambda^n (compact FP64; may not alias the
 *               inputs).
 * The forward step is recomputed from d_state_n inside the call; the grid's
 * own state and time are not changed. On a GKS_FP32C grid the recomputed
 * step is the FP32C step (d_state_n split into hi + lo as gks_set_state
 * does) and its reverse is the FP32 reverse of the recorded steps, whatever
 * the adjoint precision. Requires a fixed time step,
 * at most one rotor (with or without the velocity and tip corrections), and immersed
 * bodies only with a fixed iteration count (tol = 0) (GKS_ERR_STATE
 * otherwise), and fewer than 2^31 / 64 faces per direction (GKS_ERR_ARG
 * otherwise). Synchronises the stream. */
int gks_adjoint_workspace_bytes(const gks_grid *g, size_t *bytes);
/* Arithmetic of the local reverse maps of gks_step_adjoint (the reverse of
 * the Gauss-point flux, of the WENO5 pair, equilibrium state and normal slope,
 * and the transposed tangential passes): GKS_FP64 (default) or GKS_FP32C for
 * FP32 arithmetic. Either way the forward step is recomputed in FP64, the
 * adjoints are stored and summed in FP64, and WENO5 stencils enter FP32 as
 * differences from their centre cell. GB300 runs FP32 at about 64x the FP64
 * rate. Returns GKS_ERR_ARG for another value. */
int gks_set_adjoint_precision(gks_grid *g, int precision);
int gks_step_adjoint(gks_grid *g, void *d_adj_work, double t_n, const double *d_state_n,
                     const double *d_adj_np1, double *d_adj_n, double power_seed,
                     double *h_grad_scales, double *h_grad_uinf);

/* Recorded steps: the same reverse as gks_step_adjoint, split into a forward
 * step that keeps what its reverse reads (a "tape") and the reverse from that
 * tape, so that a checkpointed gradient runs each step forward once in the
 * backward pass instead of twice.
 *   gks_adjoint_tape_bytes     bytes of one step's tape: t_n and dt, the
 *                              ghost-filled W^n and W*, the state before the
 *                              forcing, and per stage and direction the 64
 *                              Gauss-point inputs of every face, stored in
 *                              the compute type of the reverse (about 3.2 KB
 *                              per cell with the FP64 adjoint precision,
 *                              1.7 KB with FP32);
 *   gks_adjoint_scratch_bytes  bytes of the scratch of gks_step_reverse
 *                              (the workspace of gks_step_adjoint is a tape
 *                              followed by a scratch);
 *   gks_step_record            one step of the grid exactly as gks_step(g, 1,
 *                              t_out), which also fills d_tape (device,
 *                              caller-owned, 256-byte aligned);
 *   gks_step_reverse           from the tape of step n and lambda^{n+1}
 *                              (device, compact FP64), writes lambda^n
 *                              (device, compact FP64, may not alias) and adds
 *                              the force-scale and inflow-speed gradients of
 *                              step n as gks_step_adjoint does; power_seed is
 *                              dJ/dP for the power of step n. The reverse
 *                              only reads the tape, so one tape serves any
 *                              number of reverses (several adjoint seeds); a
 *                              tape that was not recorded gives
 *                              GKS_ERR_STATE. d_scratch: device,
 *                              caller-owned, 256-byte aligned. Synchronises
 *                              the stream.
 * Both need what gks_step_adjoint needs (GKS_ERR_STATE / GKS_ERR_ARG
 * otherwise), except that they also take GKS_FP32C grids and immersed
 * bodies with a residual tolerance (the tape keeps the iterations each body
 * ran; at most 28 bodies), and use the grid's adjoint precision; a tape
 * recorded with the other precision gives GKS_ERR_STATE. The grid's force scales
 * and inflow must be those of the recorded step when it is reversed. */
int gks_adjoint_tape_bytes(const gks_grid *g, size_t *bytes);
int gks_adjoint_scratch_bytes(const gks_grid *g, size_t *bytes);
int gks_step_record(gks_grid *g, void *d_tape, double *t_out);
int gks_step_reverse(gks_grid *g, void *d_tape, void *d_scratch, const double *d_adj_np1,
                     double *d_adj_n, double power_seed, double *h_grad_scales,
                     double *h_grad_uinf);

/* Kernel accounting of the library's own kernels. Every kernel launch is
 * counted per group (0 prep, 1 ghost, 2 cfl, 3 face_eq, 4 face_flux: x and
 * y faces, 5 flux_update: z faces fused with the stage update, 6 alm, 7 ibm,
 * 8 misc); with timing enabled each launch is also
 * bracketed by CUDA events on the grid's stream and its duration summed.
 * gks_profile_enable sets timing on or off and clears the counters;
 * gks_profile_read synchronises, fills out and clears the counters. With
 * the environment variable GKS_NVTX=1 at grid creation every launch is also
 * an NVTX range named after its group (for Nsight tools). */
#define GKS_NUM_KERNEL_GROUPS 9
typedef struct {
    long launches[GKS_NUM_KERNEL_GROUPS];
    double ms[GKS_NUM_KERNEL_GROUPS];
    long total_launches;
} gks_profile_out;
int gks_profile_enable(gks_grid *g, int timing_on);
int gks_profile_read(gks_grid *g, gks_profile_out *out);
const char *gks_kernel_group_name(int group);

/* gks_diagnostics_noalloc: the same FP64 sums as gks_diagnostics (mass,
 * momentum, kinetic energy, with cell volumes), for callers that cannot
 * allocate device memory -- for example an application that owns all device
 * memory through its own pool and does not let libraries allocate, or a
 * process whose device-memory budget is already fully committed. The paper
 * has no counterpart to this call. It allocates nothing: its scratch (one
 * partial sum per block of 4096 cells) lives in a static device array of
 * 512 KiB inside the library, which every GPU that loads the library holds
 * until the process exits.
 *   d_state    device, 4 * N FP64 values (rho, rho U, rho V, rho W),
 *              component-major, x fastest, N = nx ny nz (the layout of
 *              gks_set_state, in device memory).
 *   d_hx/hy/hz device, nx / ny / nz cell widths.
 *   d_out      device, 5 doubles written by the call.
 *   stream     cudaStream_t (as void*), NULL = legacy default stream.
 * Returns GKS_ERR_ARG for null pointers, empty extents or more than
 * 33,554,432 cells (the scratch limit), GKS_ERR_CUDA if a launch fails; the
 * message is in gks_last_error(NULL). The work is asynchronous on stream.
 * Each call outside stream capture looks up the device address of the
 * static scratch (cudaGetSymbolAddress) with the current device, so a device
 * reset never leaves a stale address; a call made while its stream is being
 * captured reuses the address of the last uncaptured call on that device, so
 * make one call before any capture (and again after a device reset):
 * otherwise the captured call returns GKS_ERR_STATE. All calls share the one
 * scratch array:
 * calls that overlap on the GPU (in flight on different streams at once)
 * race and must be serialised by the caller. */
int gks_diagnostics_noalloc(const double *d_state, int nx, int ny, int nz, const double *d_hx,
                            const double *d_hy, const double *d_hz, double *d_out, void *stream);

/* gks_alu_peak_probe: a measurement aid with no counterpart in the paper.
 * Launches, asynchronously on stream, a loop of independent fused multiply-
 * adds over 4 blocks of 256 threads per SM, each thread doing iters x 128
 * FMAs, and writes to *flops the operations of that launch (2 per FMA).
 *   kind    0: FP32 FMAs; 1: FP64 FMAs; 2: FP32 FMAs as packed pairs (two
 *           lanes per FFMA2 instruction, the form of the packed stencil code).
 * Timed with CUDA events on the same stream, the ratio is the arithmetic peak
 * the stencil kernels' ALU roofline is measured against.
 *   d_sink  device buffer of at least 4 x (number of SMs) doubles; nothing is
 *           written to it in practice (it keeps the loop's result alive).
 * Returns GKS_ERR_ARG for null pointers, iters < 1 or another kind,
 * GKS_ERR_CUDA if the launch fails. */
int gks_alu_peak_probe(int kind, long iters, void *d_sink, void *stream, double *flops);

#ifdef __cplusplus
}
#endif

#endif /* GKS_API_H */
