/*
 * wsi.h -- C ABI of libwsi: the implicit Stokes step of the DLM level-set
 * wave-structure-interaction method of Nangia, Patankar & Bhalla
 * (arXiv 1901.07892) on one GB300 GPU (sm_103a), uniform staggered grid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  nx x ny x nz cells over [0,lx] x [0,ly] x [0,lz] (Sec. 3.1).  A 2-D
 *   problem is nz = 1 with free-slip z walls (bc[4] = bc[5] = +1); every
 *   z-derivative then vanishes and all w-faces lie on walls.
 * Layout.  Every array is float64, x fastest, unghosted:
 *     cell field   nx*ny*nz                 index (k*ny + j)*nx + i
 *     u (x-faces)  (nx+1)*ny*nz             index (k*ny + j)*(nx+1) + i
 *     v (y-faces)  nx*(ny+1)*nz             index (k*(ny+1) + j)*nx + i
 *     w (z-faces)  nx*ny*(nz+1)             index (k*ny + j)*nx + i
 *   A "Stokes vector" is u, v, w, p concatenated (wsi_stokes_size() doubles);
 *   a "velocity vector" is its first three parts (wsi_velocity_size()).
 *   Faces lying on a wall carry the zero normal velocity; they are not
 *   unknowns and every output writes 0 there.
 * Memory.  Array arguments may be device pointers or host pointers (pageable
 *   or pinned): the library copies with cudaMemcpyDefault on its stream.
 *   The caller keeps ownership of everything it passes; the library copies
 *   what it needs and never keeps a caller pointer after returning.
 *   The context owns all device state it allocates, on the stream given at
 *   creation; every call is stream-ordered and returns after the stream has
 *   been synchronised unless stated otherwise.
 * Errors.  Every int-returning call returns WSI_OK or one of the codes
 *   below, never aborts, and leaves a message in wsi_last_error(ctx).
 *   Device-side bound checks raise a flag read back as WSI_ERR_DEVICE (the
 *   marker update of wsi_step checks that every marker stays in the box).
 */
#ifndef WSI_H
#define WSI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WSI_OK 0
#define WSI_ERR_INVALID_ARG 1
#define WSI_ERR_CUDA 2
#define WSI_ERR_NOT_CONVERGED 3
#define WSI_ERR_NAN 4
#define WSI_ERR_OOM 5
#define WSI_ERR_DEVICE 6

#define WSI_NO_SLIP (-1.0)
#define WSI_FREE_SLIP (1.0)

#define WSI_PREC_FP64 0   /* preconditioner in float64 (plain path)           */
#define WSI_PREC_MIXED 1  /* preconditioner in float32 inside float64 FGMRES */

#define WSI_FORM_CONSISTENT 0      /* SSP-RK3 mass transport, consistent momentum
                                      convection (Sec. 4.2.2; the default)    */
#define WSI_FORM_NONCONSERVATIVE 1 /* level-set face density, explicit CUI
                                      convection N(u^{n+1/2}) (Sec. 4.2.3)    */

#define WSI_SMOOTH_RBGS 0          /* red-black Gauss-Seidel (the default)    */
#define WSI_SMOOTH_CHEBYSHEV 1     /* Chebyshev polynomial of the Jacobi-
                                      preconditioned operator, interval
                                      [1/4, 2] (Gershgorin bound 2)           */

#define WSI_LIMIT_CUI 0            /* level-set face values: bounded cubic
                                      upwind (the default stand-in)          */
#define WSI_LIMIT_XSPPM7 1         /* xsPPM7 (Sec. 4.2.1): seventh-order
                                      upwind-biased interpolant within the
                                      monotonicity-preserving, extremum-
                                      sensitive bounds of Suresh and Huynh   */

#define WSI_GRAVITY_FLOW 0 /* rho^flow g: well-balanced, for locked bodies (Sec. 5) */
#define WSI_GRAVITY_FULL 1 /* rho g with the transported face density           */

typedef struct wsi_ctx wsi_ctx;

typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    double bc[6];        /* tangential ghost sign per wall x-,x+,y-,y+,z-,z+:
                            WSI_NO_SLIP or WSI_FREE_SLIP                      */
    double gravity[3];
    double n_cells;      /* Heaviside half-width in cells (paper: 2)          */
    double theta;        /* implicit viscous weight (paper: 1/2, Crank-Nicolson) */
    int precision;       /* WSI_PREC_FP64 or WSI_PREC_MIXED                  */
    int mg_pre, mg_post; /* pressure smoothing per level and side: sweeps
                            (red-black) or polynomial degree (Chebyshev)     */
    int mg_cycles;       /* pressure V-cycles per preconditioner application  */
    int visc_sweeps;     /* viscous red-black sweeps per application (and per
                            level and side of a viscous V-cycle)              */
    int restart;         /* FGMRES restart length m                           */
    int visc_mg;         /* viscous V-cycles per application; 0: visc_sweeps
                            sweeps on the fine grid only                      */
    int reinit_iters;    /* pseudo-time steps of the level-set
                            reinitialisation at the end of every wsi_step
                            (Sec. 4.1); 0: phi is not reinitialised          */
    int transport_form;  /* WSI_FORM_CONSISTENT or WSI_FORM_NONCONSERVATIVE
                            (the formulation wsi_step integrates)            */
    int mg_smoother;     /* WSI_SMOOTH_RBGS or WSI_SMOOTH_CHEBYSHEV: smoother
                            of the pressure multigrid                        */
    int ls_limiter;      /* WSI_LIMIT_CUI or WSI_LIMIT_XSPPM7: face values of
                            the level-set advection (Sec. 4.2.1)             */
    int open_top;        /* 1: the z+ side is open (Sec. 7.1's tank: zero
                            tangential velocity and zero pressure on the top
                            plane; its z-faces are unknowns, dw/dz = 0 there).
                            Needs bc[5] = WSI_NO_SLIP, nz >= 2 and
                            visc_mg = 0; 0: a wall like the other sides      */
} wsi_grid_desc;

typedef struct {
    double rho_l, rho_g, rho_s;
    double mu_l, mu_g, mu_s;
    int gravity_mode;    /* WSI_GRAVITY_FLOW or WSI_GRAVITY_FULL             */
} wsi_phase_props;

typedef struct {
    const double* X;     /* marker positions, n_markers x 3 (x,y,z interleaved) */
    int n_markers;
    double dV;           /* marker volume ds1 ds2 ds3                         */
    int lock[6];         /* 1 = prescribed: Ux,Uy,Uz,Wx,Wy,Wz                 */
    double U_pres[3], W_pres[3];
    int shape;           /* psi rebuilt each cycle as the signed distance about
                            the markers' mean (Sec. 4.1): 0 none (psi kept);
                            1 box of half-extents half[0..2]; 2 cylinder with
                            its axis along y, radius half[0], half length
                            half[1]                                         */
    double half[3];
} wsi_body_desc;

typedef struct {
    double rtol;         /* relative residual ||b-Kx||_2 / ||b||_2            */
    int max_iters;
    int use_x0;          /* 1: x holds the initial guess                      */
} wsi_solve_opts;

typedef struct {
    int iters;
    double rel_residual; /* true residual after the solve                      */
    double ms;
    int learned_rejected; /* wsi_pressure_solve: cycle whose learned correction
                             was undone (-1: none); else -1                   */
    int guess;           /* wsi_pressure_solve with a guess network: 1 its
                            initial guess was kept, 0 it was dropped (its
                            residual was not below the zero guess's); else -1 */
} wsi_solve_stats;

typedef struct {
    double U_r[3], W_r[3], X_com[3];
} wsi_body_state;

typedef struct {
    int iters[4];        /* FGMRES iterations of each cycle's solve           */
    double rel_residual[4];
    double umax;         /* max |u| over all faces after the step              */
    double ms;
    double F_lm[3];      /* net hydrodynamic force on the body by the Lagrange-
                            multiplier method (Sec. 8): sum over the markers of
                            rho_s [(U_b^{n+1} - U_b^n) - dU^{n+1}] dV / dt with
                            dU = U_b - J u~ of the last cycle; 0 without a
                            body                                              */
} wsi_step_stats;

/* Sizes of the packed vectors (doubles). */
size_t wsi_stokes_size(const wsi_ctx* ctx);
size_t wsi_velocity_size(const wsi_ctx* ctx);

/* Create a context: grid, boundary conditions, solver options (Sec. 3.1 grid,
 * Sec. 4.2.4 solver).  stream: a cudaStream_t (NULL = legacy default stream).
 * The device is the current one.  *out is owned by the caller until
 * wsi_destroy.  WSI_ERR_INVALID_ARG on non-positive sizes or spacings, or
 * a grid with (nx+1)(ny+1)(nz+1) >= 2^31 (32-bit array offsets). */
int wsi_create_grid(const wsi_grid_desc* desc, void* stream, wsi_ctx** out);
void wsi_destroy(wsi_ctx* ctx);
const char* wsi_last_error(const wsi_ctx* ctx);

/* Set the level sets phi (liquid-gas, liquid where phi < 0) and psi (solid,
 * inside where psi < 0) at cell centres, the material constants and the
 * bodies; compute the material coefficients of Sec. 4.1 (smoothed Heaviside
 * over n_cells cells, two-stage property, harmonic edge viscosity) and the
 * face density from face-averaged level sets (Sec. 4.2.2).  Resets the
 * velocity history to zero.  Markers are copied in.  WSI_ERR_INVALID_ARG on
 * non-finite or non-positive material constants, n_bodies > 1, or a marker
 * outside the box. */
int wsi_set_phases(wsi_ctx* ctx, const double* phi, const double* psi,
                   const wsi_phase_props* props, const wsi_body_desc* bodies, int n_bodies);

/* Solve the implicit Stokes system of Sec. 4.2.2 / 4.2.4,
 *     rho/dt u - theta L_mu u + G p = b_u,   -D u = b_p,
 * with the coefficients of the last wsi_set_phases, by FGMRES(m)
 * right-preconditioned with the projection method (viscous red-black
 * smoothing, pressure multigrid V-cycles).  rhs, x: Stokes vectors; x is
 * the initial guess when opts->use_x0, and receives the solution with p of
 * zero mean.  Returns WSI_ERR_NOT_CONVERGED (solution still written) when
 * max_iters is reached, WSI_ERR_NAN on a non-finite residual. */
int wsi_stokes_solve(wsi_ctx* ctx, const double* rhs, double* x, double dt,
                     const wsi_solve_opts* opts, wsi_solve_stats* stats);

/* Rigidity projection of Sec. 4.2.5 for the body of the last
 * wsi_set_phases at its current markers: U = J u, free DOFs from momentum
 * redistribution, locked DOFs prescribed, U_b = U_r + W_r x R,
 * u += S(U_b - U), with the wall-adjoint J_BC / S_BC of Sec. 3.3.2.
 * vel: velocity vector, corrected in place.  Markers do not move. */
int wsi_dlm_constrain(wsi_ctx* ctx, double* vel, wsi_body_state* out);

/* One full time step of Sec. 4.2 (two fixed-point cycles): level-set
 * advection, psi rebuilt from the markers, materials, SSP-RK3 face density
 * and consistent convection, Stokes solve, rigidity projection and marker
 * update, on library-owned state.  With transport_form =
 * WSI_FORM_NONCONSERVATIVE the momentum equation of Sec. 4.2.3 replaces the
 * consistent one: rho^{n+1,k+1} (u - u^n)/dt + rho^{n+1,k+1} N = -G p +
 * L_mu u (same Crank-Nicolson split) + rho_g g, with rho^{n+1,k+1} the face
 * density of the level sets and N the CUI-limited div(u^{n+1/2,k} u) (no mass
 * transport).  Tolerance and limits from opts.
 * WSI_ERR_DEVICE when the device bound check of the marker update saw a
 * marker leave the box by more than half a cell or turn non-finite; the step
 * is then committed as computed and the flag cleared, so the caller decides
 * whether to go on. */
int wsi_step(wsi_ctx* ctx, double dt, const wsi_solve_opts* opts, wsi_step_stats* stats);

/* State access for the step.  which: WSI_F_VEL (velocity vector u^n;
 * setting it also sets u^{n-1} = u^n), WSI_F_VEL_OLD (u^{n-1}, used by the
 * extrapolated transport velocities of Sec. 4.2.2), WSI_F_P (cell),
 * WSI_F_PHI, WSI_F_PSI (cell), WSI_F_MARKERS (n x 3, get only). */
#define WSI_F_VEL 0
#define WSI_F_P 1
#define WSI_F_PHI 2
#define WSI_F_PSI 3
#define WSI_F_MARKERS 4
#define WSI_F_VEL_OLD 5
int wsi_get_field(wsi_ctx* ctx, int which, double* dst);
int wsi_set_field(wsi_ctx* ctx, int which, const double* src);

/* Checkpoint / restart of the time-stepping state (no counterpart in the
 * paper): u^n, u^{n-1}, p, phi, psi, the markers, their velocity U_b^n, the
 * body's rigid velocities and centre, the time and the static-psi flag, and
 * with a Dirichlet inlet the tangential inlet data of u^n and u^{n-1}, to a
 * host file (native byte order).  wsi_restore needs a context created with
 * the same grid and precision, wsi_set_phases with the same body and, for a
 * checkpoint with an inlet, wsi_set_waves with the same inlet (the phase
 * properties, body and wave descriptions are not stored); it recomputes the
 * operator coefficients from the restored level sets, so that stepping on
 * continues exactly as without the interruption.  Errors:
 * WSI_ERR_INVALID_ARG (no phases, unreadable file, other grid), WSI_ERR_CUDA. */
int wsi_checkpoint(wsi_ctx* ctx, const char* path);
int wsi_restore(wsi_ctx* ctx, const char* path);

/* Coefficients computed by wsi_set_phases (Sec. 4.1): which:
 * WSI_C_RHO_CC, WSI_C_MU_CC (cell), WSI_C_RHO_FACE, WSI_C_RHO_FLOW_FACE
 * (velocity vectors), WSI_C_MU_EDGE (mu_xy, mu_xz, mu_yz concatenated:
 * (nx+1)(ny+1)nz + (nx+1)ny(nz+1) + nx(ny+1)(nz+1)). */
#define WSI_C_RHO_CC 0
#define WSI_C_MU_CC 1
#define WSI_C_RHO_FACE 2
#define WSI_C_RHO_FLOW_FACE 3
#define WSI_C_MU_EDGE 4
int wsi_get_coeff(wsi_ctx* ctx, int which, double* dst);

/* Operator applies on the current coefficients (float64), Sec. 3.1 and
 * Sec. 4.2.2:  WSI_OP_STOKES  Stokes vector -> Stokes vector (K x);
 * WSI_OP_VISCOUS  velocity -> velocity (rho/dt u - theta L_mu u);
 * WSI_OP_STRAIN  velocity -> velocity (L_mu u);
 * WSI_OP_PRESSURE cell -> cell (D beta G p, beta = 1/rho face);
 * WSI_OP_GRAD cell -> velocity; WSI_OP_DIV velocity -> cell. */
#define WSI_OP_STOKES 0
#define WSI_OP_VISCOUS 1
#define WSI_OP_STRAIN 2
#define WSI_OP_PRESSURE 3
#define WSI_OP_GRAD 4
#define WSI_OP_DIV 5
int wsi_apply(wsi_ctx* ctx, int op, const double* in, double* out, double dt);

/* Consistent transport of Sec. 4.2.2 on the current face density rho^n:
 * SSP-RK3 with u^n, u^(1), u^(2) for cycle k (u_k = u^{n+1,k}, ignored at
 * k = 0) -> rho_out (velocity-vector layout) and the convective term C_out. */
int wsi_transport(wsi_ctx* ctx, const double* u_n, const double* u_nm1, const double* u_k,
                  int k, double dt, double* rho_out, double* C_out);

/* Level-set advection of Sec. 4.2.1: phi_out = phi_n - dt div(u phi_lim(phi_half)). */
int wsi_advect_levelset(wsi_ctx* ctx, const double* vel, const double* phi_n,
                        const double* phi_half, double dt, double* phi_out);

/* Reinitialisation of the flow level set (Sec. 4.1): iters steps of the
 * eikonal equation  d phi/d tau + sgn(phi~)(|grad phi| - 1) = 0  from
 * phi~ = phi, with second-order ENO one-sided differences, the subcell fix
 * of Min (2010) where phi~ changes sign between neighbours (the interface at
 * the zero of the quadratic through phi~, phi = 0 there), the Godunov
 * Hamiltonian of sgn(phi~), two-stage TVD Runge-Kutta with the local step
 * 0.3 min(h, subcell distances), and Neumann mirror ghosts.  sgn(phi~) and
 * the subcell distances stay fixed (immobile interface).  phi: cells
 * (Nx Ny Nz doubles, x fastest, host or device), updated in place.
 * Arithmetic in float64 (WSI_PREC_FP64) or float32 (WSI_PREC_MIXED, the
 * change then added to the float64 input).  WSI_ERR_INVALID_ARG for a null
 * phi or iters < 0; iters = 0 leaves phi unchanged. */
int wsi_reinit(wsi_ctx* ctx, double* phi, int iters);

/* IB4 transfers of Sec. 3.3 with the wall-adjoint forms of Sec. 3.3.2.
 * X: n x 3 positions.  interp: velocity vector -> U (n x 3).
 * spread: F (n x 3), marker volume dV -> velocity vector (overwritten). */
int wsi_interp(wsi_ctx* ctx, const double* vel, const double* X, int n, double* U);
int wsi_spread(wsi_ctx* ctx, const double* F, const double* X, int n, double dV, double* vel);

/* Numerical wave tank of Sec. 7.1: second-order Stokes wave of height H,
 * period T over still-water depth `depth` (dispersion omega^2 = g k tanh kd
 * solved by Newton's method; g = |gravity|).  At the end of every wsi_step
 * the velocity and phi are relaxed, q <- a q + (1-a) q_target with
 * a = 1 - (exp(xb^3.5) - 1)/(e - 1), in a generation zone [0, x_gen]
 * (targets: phi = y - eta, liquid-only Stokes velocity) and a damping zone
 * [x_damp, lx] (targets: still water), y = height above still water along
 * axis `vertical` (1 or 2).  t0 sets the time of the current state; each
 * step advances it by dt.  NULL disables the zones.
 * wsi_wave_relax applies one relaxation at time t to a velocity vector and
 * (optionally, phi may be NULL) a cell field, in place. */
typedef struct {
    double H, T, depth;
    double x_gen, x_damp;
    double t0;
    int vertical;
    int inlet;           /* 1: Dirichlet wave inlet on the x- plane (Sec. 7.1):
                            the x- faces carry the liquid-only normal Stokes
                            velocity (1 - H~(phi_b)) u_w(0, z, t), phi_b =
                            z - d - eta(0, t), and the x- edges the vertical
                            one, imposed through the ghost 2 w_b - w; the data
                            of t^{n+1} are lifted into the implicit solve.
                            Needs vertical = 2 and bc[0] = WSI_NO_SLIP; x_gen
                            may then be 0 (no generation zone).  Sets the x-
                            faces of the current velocity and of the previous
                            one to the data of t0: set the state first      */
} wsi_wave_desc;
int wsi_set_waves(wsi_ctx* ctx, const wsi_wave_desc* w);
int wsi_wave_relax(wsi_ctx* ctx, double t, double* vel, double* phi);

/* Learned pressure correction (no counterpart in the paper: it extends the
 * pressure multigrid of the projection preconditioner).  A 3-D U-Net of
 * widths c0/c1/c2 (multiples of 16, c0 <= 16, c1 <= 32, c2 <= 64) on a grid
 * of nz x ny x nx cells (each divisible by 4): per level two 3x3x3
 * convolutions with ReLU, 2x2x2 average pooling down, nearest up-sampling with
 * skip concatenation up, a 1x1x1 head to one channel.  BF16 weights and
 * activations; each 3x3x3 convolution (forward, and the input-gradient
 * pass) is an implicit GEMM on the fifth-generation tensor cores
 * (tcgen05.mma, float32 accumulator in tensor memory); float32 master
 * weights and Adam.  Parameters are one float32 vector: per convolution
 * (a1 a2 b1 b2 c1 c2 ub1 ub2 ua1 ua2) weights [27 taps][C_out][C_in]
 * (tap = 9 dz + 3 dy + dx; a1's C_in is padded from 3 to 16) then biases
 * [C_out]; then the head's weights [c0] and bias.
 * wsi_unet_create initialises the weights from `seed` (He normal).
 * wsi_unet_forward: x [V][3] float32 (host or device) -> out [V].
 * wsi_unet_backward (after a forward): gradients of 0.5 mean((out - t)^2),
 * readable with wsi_unet_get_grads; wsi_unet_adam applies one Adam step
 * (beta 0.9 / 0.999).  Forward and backward return WSI_ERR_DEVICE when a
 * convolution's bounded wait for the tensor core ran out (its outputs are
 * then not valid; nothing traps). */
typedef struct wsi_unet wsi_unet;
int wsi_unet_create(int nz, int ny, int nx, int c0, int c1, int c2, unsigned long long seed, wsi_unet** out);
void wsi_unet_destroy(wsi_unet* net);
size_t wsi_unet_num_params(const wsi_unet* net);
int wsi_unet_set_params(wsi_unet* net, const float* p);
int wsi_unet_get_params(wsi_unet* net, float* p);
int wsi_unet_get_grads(wsi_unet* net, float* g);
int wsi_unet_forward(wsi_unet* net, const float* x, float* out);
int wsi_unet_backward(wsi_unet* net, const float* target, double* loss);
int wsi_unet_adam(wsi_unet* net, double lr);

/* Use `net` in the float32 pressure multigrid at hierarchy level `level`
 * (1 = first coarsening; the net's grid must equal that level's).
 * enable = WSI_LEARN_REPLACE: the V-cycle replaces everything below the level
 * by the network's prediction for the level's right-hand side, followed by
 * post-smoothing.  enable = WSI_LEARN_AUGMENT: the plain coarse-grid
 * correction runs, then the network's prediction for the level's residual is
 * added before post-smoothing.  enable = WSI_LEARN_OFF keeps it attached but
 * unused.  Inputs: log(rho)/7 and the level set averaged down to the level,
 * and the right-hand side (or residual) over its RMS; the prediction o gives
 * the correction s o / d (s the RMS, d the level operator's diagonal).
 * Requires a WSI_PREC_MIXED context and wsi_set_phases.
 * wsi_unet_train_sample: one Adam step (learning rate lr; lr = 0 only
 * evaluates) on the exact pair built from a smooth field e given on the
 * level's cells (float64, x fastest): right-hand side r = L e with solution
 * e for the replacing mode; for the augmenting mode the plain coarse-grid
 * correction x1 of r is run first and the pair is (r - L x1, e - x1).  The
 * mode is the one last given to wsi_attach_unet (WSI_LEARN_OFF trains the
 * replacing mode).  The loss is what the plain cycle judges a correction by:
 * 1/2 mean((L t)^2)/s^2 + 0.05 mean((d t)^2)/s^2 with t the error of the
 * corrected iterate; *loss receives it. */
/* Network weights and Adam state to / from a file (float32, native byte
 * order, with a header of the widths; a net of other widths is rejected with
 * WSI_ERR_INVALID_ARG).  The grid size is not stored: weights of one net
 * load into a net of any size with the same widths. */
int wsi_unet_save(wsi_unet* net, const char* path);
int wsi_unet_load(wsi_unet* net, const char* path);

enum { WSI_LEARN_OFF = 0, WSI_LEARN_REPLACE = 1, WSI_LEARN_AUGMENT = 2 };
int wsi_attach_unet(wsi_ctx* ctx, wsi_unet* net, int level, int enable);
int wsi_unet_train_sample(wsi_ctx* ctx, const double* e, double lr, double* loss);

/* Learned initial guess for wsi_pressure_solve (an extension of the
 * learned pressure part: the network supplies the solve's starting iterate;
 * not in the paper).
 * wsi_attach_unet_guess: a network sized for multigrid level `level` of this
 * (WSI_PREC_MIXED) context, or NULL to detach.  Its input is the level's
 * restriction (cell averages) of the right-hand side with log rho and phi
 * (as for wsi_attach_unet); its output o gives the level's solution
 * G s o / d (G = (n_max/pi)^2, n_max the level's longest extent in cells),
 * prolongated to the fine grid as the initial iterate, which is kept only if
 * its residual is below the zero guess's (wsi_solve_stats.guess).
 * wsi_unet_train_guess: one Adam step (lr = 0: evaluate) on a pair the
 * solver generated: a fine right-hand side y and its solution x (cell
 * fields, float64, host or device, x fastest); both are averaged down to the
 * level and the loss 1/2 mean((o - d x_l / (G s))^2) is written to *loss. */
int wsi_attach_unet_guess(wsi_ctx* ctx, wsi_unet* net, int level);
int wsi_unet_train_guess(wsi_ctx* ctx, const double* y, const double* x, double lr, double* loss);

/* Standalone pressure solve D(beta G) x = y (Sec. 4.2.4's projection
 * sub-problem) on the current coefficients: float64 residuals with
 * multigrid V-cycle corrections (float32 cycles on WSI_PREC_MIXED contexts,
 * with the attached network if enabled; float64 on WSI_PREC_FP64), until
 * ||y - L x|| <= rtol ||y|| (y's mean removed; x of zero mean).  A learned
 * cycle that fails to reduce the residual switches the rest of the solve to
 * plain cycles.  stats->iters = V-cycles. */
int wsi_pressure_solve(wsi_ctx* ctx, const double* y, double* x, double rtol, int max_cycles,
                       wsi_solve_stats* stats);

/* Float64 2-norm sqrt(sum x_i^2) of n doubles at device pointer x, written
 * to *out (host or device pointer) before the call returns; deterministic
 * (fixed reduction tree).  The paper has no counterpart: this is the
 * allocation-free variant of the reductions the solver runs on its own
 * scratch, for callers that must not allocate device memory after set-up.
 * Its scratch is static device memory (64 KiB of partial sums), so it
 * allocates nothing; the first call on a device does the set-up (looks up
 * that memory) and should come before any stream capture; first calls from
 * several host threads on one device must be serialised.  n > 2^27
 * (134,217,728) is rejected with WSI_ERR_INVALID_ARG, and so is an x that is
 * not device (or managed) memory of the current device (checked with
 * cudaPointerGetAttributes, before any launch).  Calls that can overlap
 * (other streams, host threads) share the scratch and race.  The call
 * synchronises `stream` before it returns.
 * stream: a cudaStream_t (NULL = legacy default stream). */
int wsi_norm2_noalloc(const double* x, size_t n, double* out, void* stream);

/* Instrumentation (no counterpart in the paper; used to report kernel
 * rooflines).  wsi_launch_count: kernels launched by this library in this
 * process so far.  wsi_ktimer_enable(k): bracket every later launch of
 * kernel class k with CUDA events on its own stream (k = -1 disables;
 * enabling resets the record).  wsi_ktimer_read: summed device time and
 * number of bracketed launches (synchronises on the recorded events).
 * Classes: 0 Stokes matvec, 1 pressure red-black sweep, 2 viscous red-black
 * sweep, 3 transport flux divergence, 4 Gram-Schmidt dots, 5 Gram-Schmidt
 * axpy, 6 residual restriction, 7 prolongation. */
long long wsi_launch_count(void);
int wsi_ktimer_enable(int kernel_class);
int wsi_ktimer_read(double* total_ms, long long* launches);
/* Summed algorithmic bytes of the bracketed launches of the enabled class,
 * for classes whose launches differ in size (Gram-Schmidt dots: each
 * distinct vector read once; multi-axpy: the rows and w read, w written);
 * 0 for the other classes. */
int wsi_ktimer_bytes(double* bytes);

/* Measured fused multiply-add rate of the current GPU in GFLOP/s (2 flop per
 * FMA): fp64 = 1 float64, 0 float32, 2 float32 issued as packed pairs
 * (fma.rn.f32x2, sm_100 and later); eight independent register FMA
 * chains per thread, 8 blocks of 256 threads per SM, best of three ~60 ms
 * launches after a warm-up, timed with CUDA events on `stream`.  The
 * denominator of the roofline of kernels bound by arithmetic issue.  No
 * counterpart in the paper.  Allocates (and frees) a small device buffer;
 * synchronises `stream`.  Errors: WSI_ERR_INVALID_ARG (null gflops, fp64
 * outside 0..2),
 * WSI_ERR_OOM, WSI_ERR_CUDA. */
int wsi_fma_peak(int fp64, void* stream, double* gflops);

#ifdef __cplusplus
}
#endif
#endif
