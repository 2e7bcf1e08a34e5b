/*
 * rossbi.h - C ABI of the GB300 RoSSBi3D hot-path library (librossbi.so).
 *
 * The library advances the compressible Euler + energy equations of an ideal
 * gas, coupled by aerodynamic drag to a pressureless dust fluid, on a
 * logarithmic-in-r cylindrical (r, theta, z) grid or a Cartesian Box, by the
 * method of Rendon Restrepo, Barge & Vavrik, "RoSSBi3D: a 3D and bi-fluid code
 * for protoplanetary discs" (arXiv:2207.04252):
 *   - cell-centred finite volumes on the conservative variables (Sect. 2.2,
 *     App. B order: rho u, rho v, rho w, E, rho; dust: rho_d u_d, rho_d v_d,
 *     rho_d w_d, rho_d),
 *   - parabolic reconstruction, with a MinMod limiter, of the deviation of
 *     each conservative gas variable from the equilibrium (Sect. 2.7 on the
 *     variables of App. B; the deviation of the primitive variables as an
 *     option) and of the dust's primitive variables,
 *   - an exact Riemann solver at every gas face (Sect. 2.6) and an upwind
 *     pressureless flux at every dust face (Sect. 2.9),
 *   - geometric, gravity, rotating-frame and drag sources, balanced by the
 *     empty-run residual (Sects. 2.1, 2.8, 2.9, App. B),
 *   - midpoint RK2 in time with a global CFL step (Sect. 2.5).
 *
 * Conventions shared by every entry point
 *   - All functions return a rossbi_status; none throws, traps or exits.
 *   - State arrays are caller-owned DEVICE buffers, one per field
 *     (structure of arrays), each holding nr*nth*nz values at linear index
 *     (k*nth + j)*nr + i (r fastest).  Their element type depends on the
 *     grid's precision form (see rossbi_precision).
 *   - Everything is ordered on the CUDA stream given to rossbi_init_grid.
 *     Calls that return a host value (dt, sums) synchronise that stream.
 *   - Kernels record non-physical states (rho <= 0, P <= 0, NaN) and Riemann
 *     non-convergence in a device status word; they never trap.  The word is
 *     read (and cleared) by rossbi_take_status and by every call that
 *     synchronises; a set bit turns into ROSSBI_ERR_NONPHYSICAL or
 *     ROSSBI_ERR_RIEMANN.
 *   - A grid is not thread-safe: one host thread at a time per grid.
 */
#ifndef ROSSBI_H
#define ROSSBI_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ROSSBI_OK = 0,
  ROSSBI_ERR_ARG = 1,          /* invalid argument or call order */
  ROSSBI_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  ROSSBI_ERR_OOM = 3,          /* device allocation failed */
  ROSSBI_ERR_NONPHYSICAL = 4,  /* rho <= 0, P <= 0 or NaN met by a kernel */
  ROSSBI_ERR_RIEMANN = 5,      /* star-pressure Newton iteration did not converge */
  ROSSBI_ERR_UNSUPPORTED = 6   /* valid but not implemented combination */
} rossbi_status;

enum { ROSSBI_GEOM_BOX = 0, ROSSBI_GEOM_CYL = 1 };
enum { ROSSBI_BC_PERIODIC = 0, ROSSBI_BC_OUTFLOW = 1, ROSSBI_BC_EQUILIBRIUM = 2 };

/* Precision forms.
 *   ROSSBI_FP64      : state = full conservative E, double.
 *   ROSSBI_FP32_PERT : state = deviation E' = E - E0 from the stored FP64
 *                      equilibrium, float; the update is computed in
 *                      perturbation form (see rossbi_step).
 *   ROSSBI_FP64_PERT : the perturbation form in double (state E', double). */
enum { ROSSBI_FP64 = 0, ROSSBI_FP32_PERT = 1, ROSSBI_FP64_PERT = 2 };

/* Gas reconstruction (Sect. 2.7).
 *   ROSSBI_RECON_CONSERVATIVE : the paper's scheme.  The parabola and MinMod
 *                      limiter act on each deviation E'_p = E_p - E0_p of the
 *                      conservative variables of App. B (rho u, rho v, rho w,
 *                      E, rho); a face state is E0 at the face plus the
 *                      interpolated deviation.  The default (0).
 *   ROSSBI_RECON_PRIMITIVE : the same parabola and limiter on the deviations
 *                      of the primitive variables (rho, u, v, w, P) from the
 *                      equilibrium primitives.  Not the paper's scheme: an
 *                      option for fast rotating frames and vortex runs, where
 *                      the conservative face pressure, a difference of terms
 *                      O(Mach^2) larger than itself, makes the conservative
 *                      scheme sensitive to rounding.
 * The dust is reconstructed in its primitive variables in both modes. */
enum { ROSSBI_RECON_CONSERVATIVE = 0, ROSSBI_RECON_PRIMITIVE = 1 };

typedef struct rossbi_grid rossbi_grid; /* opaque, library-owned */

/* Grid description (Sect. 2.3 mesh, Sect. 2.4 boundaries).
 *   geometry : ROSSBI_GEOM_CYL (r log-spaced on [x0[0], x1[0]], theta and z
 *              uniform) or ROSSBI_GEOM_BOX (x, y, z uniform, no sources).
 *   nr,nth,nz: cells along r (x), theta (y), z.  Each >= 1.
 *   bc_lo/hi : per axis; ROSSBI_BC_EQUILIBRIUM ghosts carry E' = 0,
 *              PERIODIC wraps, OUTFLOW copies the nearest interior E'.
 *              A cylindrical grid needs periodic theta and non-periodic r.
 *   gamma    : ratio of specific heats (> 1).
 *   gm       : G M of the central star (cylindrical only; >= 0, and > 0 for a
 *              disc equilibrium or the constant-Stokes drag law, which use
 *              the Keplerian frequency).
 *   omega_frame : angular speed of the rotating frame (cylindrical only).
 *   cfl      : N_CFL of the CFL condition (Sect. 2.5; the paper uses 1/2).
 *   n_dust   : number of pressureless dust fluids (species), 0 .. 4; the
 *              state has 5 + 4 n_dust fields, species s in fields 5 + 4 s ..
 *              8 + 4 s (rho_d u_d, rho_d v_d, rho_d w_d, rho_d).  Several
 *              species (the multi-fluid approach Sect. 5.4 names) each couple
 *              to the gas by their own drag, St x their factor
 *              (rossbi_set_dust_species); rossbi_adjoint_step takes at most
 *              one (ROSSBI_ERR_UNSUPPORTED).
 *   precision: one of the precision forms above.
 *   recon    : one of the reconstruction modes above. */
typedef struct {
  int geometry;
  int nr, nth, nz;
  double x0[3], x1[3];
  int bc_lo[3], bc_hi[3];
  double gamma, gm, omega_frame, cfl;
  int n_dust;
  int precision;
  int recon;
} rossbi_grid_desc;

/* Disc equilibrium parameters (App. A): Sigma = sigma0 r^beta_sigma,
 * T = T0 r^beta_T (k_B/(mu m_u) = 1).  Optionally the radial density bump of
 * the Rossby-wave-instability disc (Sect. 4.3) as part of the equilibrium:
 * rho and P scaled by 1 + bump_delta G(r), G = exp(-(r - bump_r0)^2 /
 * (2 bump_width^2)), at the same temperature, with v_theta in radial balance
 * with the bumped pressure (a stationary solution of its own).
 * bump_delta = 0 (zero-initialised) means no bump; otherwise
 * bump_delta > -1 and bump_width > 0. */
typedef struct {
  double sigma0, beta_sigma, T0, beta_T;
  double bump_delta, bump_r0, bump_width;
} rossbi_disc_params;

/* Drag (Sect. 2.9).  drag_law 0: t_s = stokes / Omega_K(r) (Box: t_s = stokes);
 * drag_law 1: Epstein t_s = rho_s r_p / (rho_g c_s) with rho_s r_p fixed so
 * that the Stokes number equals `stokes` at r = 1, z = 0 of the equilibrium;
 * drag_law 2: law 1 plus the Stokes regime, t_s = (4/9)(r_p / lambda) t_E
 * where r_p > 9 lambda / 4, with the mean free path lambda = lambda_0 / rho_g
 * and kappa = r_p / lambda_0 (>= 0; ignored by laws 0 and 1).  Law 2 is not
 * available to rossbi_step_noalloc (ROSSBI_ERR_ARG). */
typedef struct {
  double stokes;
  int drag_law;
  double kappa;
} rossbi_dust_params;

/* Radial wave-killing zones (Sect. 2.4 names them; the relaxation is that of
 * de Val-Borro et al. 2006): r_in <= r < r_edge_in and r_edge_out < r <= r_out.
 * period_factor scales the relaxation time, tau = period_factor x the
 * Keplerian orbital period 2 pi / Omega_K at that zone's boundary. */
typedef struct {
  double r_edge_in, r_edge_out, period_factor;
} rossbi_damping_params;

/* Vertical sheared damped boundary (Sect. 2.4 names it, after the works it
 * cites, without a formula): the equilibrium ghost cells beyond +-z_max
 * (bc ROSSBI_BC_EQUILIBRIUM in z, the sheared Keplerian flow) and, in
 * |z| > z_edge, the relaxation of the radial wave-killing zones turned
 * vertical, with tau = period_factor x the Keplerian orbital period
 * 2 pi / Omega_K(r) at the cell's radius. */
typedef struct {
  double z_edge, period_factor;
} rossbi_vertical_damping_params;

/* Creates a grid: mesh, metrics and device tables (Sects. 2.2-2.4).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream); not owned.
 * On success *out is a new grid to be freed with rossbi_destroy.
 * Errors: ROSSBI_ERR_ARG (bad desc or out == NULL), ROSSBI_ERR_OOM,
 * ROSSBI_ERR_CUDA, ROSSBI_ERR_UNSUPPORTED. */
rossbi_status rossbi_init_grid(const rossbi_grid_desc* desc, void* cuda_stream, rossbi_grid** out);

/* Sets the disc equilibrium E0 (App. A) at cell centres and faces, and runs
 * the "empty run" of Sect. 2.8 once to store the balanced residual
 * R0 = G(E0) used by the FP64 form.  disc == NULL sets E0 = 0: Box runs, and
 * cylindrical runs without a disc such as the explosion test of Sect. 4.1
 * (FP64 form only: the perturbation forms return ROSSBI_ERR_UNSUPPORTED for a
 * cylindrical grid without a disc).  Synchronises the stream. */
rossbi_status rossbi_set_equilibrium(rossbi_grid* g, const rossbi_disc_params* disc);

/* Indirect gravity of Sect. 2.10.  The star, pulled by an asymmetric disc,
 * accelerates; in its frame gas and dust feel -grad Phi_ind with
 *   grad Phi_ind = X_ref (A cos(theta) + B sin(theta), -A sin(theta) + B cos(theta), 0)
 * in (r, theta, z) components, where A and B are the integrals of
 * r cos(theta) / R^3 and r sin(theta) / R^3 (R^2 = r^2 + z^2) over the disc
 * mass.  Each RK stage sums them over the cells of its input state in FP64,
 * taking as mass V (rho - rho_0 + rho_d) at the cell centre: the
 * axisymmetric equilibrium exerts no net pull, so an undisturbed disc stays
 * exactly at equilibrium.  As in the paper the vertical component is
 * dropped.  The gas energy gains the work of the force; the balanced
 * residual R0 carries no indirect term.
 *   x_ref : X_ref, the gravitational constant in the code units in which
 *           density times volume is mass; 0 switches the term off (the
 *           default).  Finite; non-zero only on cylindrical grids.
 * The first non-zero call allocates (and synchronises) the device tables;
 * later calls only change the constant.  While the term is on, each step
 * launches a moments kernel and its reduction before each stage, and
 * rossbi_adjoint_step carries the term too: its local part, and the
 * cotangent that reaches every cell's rho and rho_d through A and B (one
 * more reduction and broadcast per stage).
 * Errors: ROSSBI_ERR_ARG (NULL grid, non-finite x_ref, non-zero x_ref on a
 * Box), ROSSBI_ERR_OOM, ROSSBI_ERR_CUDA. */
rossbi_status rossbi_set_indirect(rossbi_grid* g, double x_ref);

/* Wave-killing zones at the radial edges (Sect. 2.4).  Inside a zone the
 * five conservative gas departures relax towards the equilibrium,
 *   dE'/dt = -E' R(r) / tau,
 * with R(r) the parabola that is 1 at the domain boundary and 0, with zero
 * slope, at the zone's edge (rates tabulated at cell centres).  The term is
 * part of G, so it acts inside both RK stages and in rossbi_adjoint_step.
 * Dust is not damped.  p == NULL switches the zones off (the default);
 * otherwise r_in < r_edge_in <= r_edge_out < r_out and period_factor > 0.
 * Cylindrical grids with a disc equilibrium only.  Allocates an nz x nr
 * rate table (shared with the vertical damped boundary); synchronises the
 * stream.
 * Errors: ROSSBI_ERR_ARG, ROSSBI_ERR_OOM, ROSSBI_ERR_CUDA. */
rossbi_status rossbi_set_damping(rossbi_grid* g, const rossbi_damping_params* p);

/* Halo exchange of a decomposition in theta.  Sect. 3.1 splits the grid
 * into blocks that exchange ghost cells with their neighbours; a sub-domain
 * here is a grid of its own whose theta extent is its owned rows plus four
 * halo rows on each side (two per RK stage: the step's E* must be right two
 * rows beyond the owned ones), with the same dtheta as the whole grid, and
 * every step is followed by an exchange of those halo rows.  These two calls
 * move the rows: pack copies rows j0 .. j0 + rows - 1 of every field of the
 * state into buf, unpack copies buf into those rows.
 *   state : nfields device pointers of the grid's precision form.
 *   buf   : device buffer of nfields * nz * rows * nr elements of the state's
 *           type, laid out [field][k][row][i] (contiguous; on several GPUs it
 *           is what a neighbour sends or receives).
 *   0 <= j0, j0 + rows <= nth, rows >= 1.
 * One kernel launch on the grid's stream; asynchronous.
 * Errors: ROSSBI_ERR_ARG, ROSSBI_ERR_CUDA. */
rossbi_status rossbi_pack_theta_rows(rossbi_grid* g, const void* const* state, int j0, int rows, void* buf);
rossbi_status rossbi_unpack_theta_rows(rossbi_grid* g, void* const* state, int j0, int rows, const void* buf);

/* Stokes numbers of several dust species (Sect. 5.4's multi-fluid approach;
 * the drag law of Sect. 2.9 applies to each species).  Species s has the
 * Stokes number St x stokes_factor[s], St that of rossbi_dust_params; under
 * the Epstein laws its rho_s r_p scales the same way.
 *   stokes_factor : host array of n = n_dust doubles; stokes_factor[0] must be
 *                   1 (species 0 has St itself), the others > 0 and finite.
 * The drag of n_dust > 1 species is the closed-form solution of the
 * backward-Euler system that couples the gas to every species (no
 * dust-dust exchange): v_g' = (rho_g v_g + sum rho_k w_k v_k) /
 * (rho_g + sum rho_k w_k), v_k' = (v_k + a_k v_g') / (1 + a_k), a_k = tau /
 * t_k, w_k = a_k / (1 + a_k); the gas energy gains the drag's work.
 * Default: every factor 1.  Takes effect from the next step.
 * Errors: ROSSBI_ERR_ARG (NULL, n != n_dust, n_dust = 0, a bad factor). */
rossbi_status rossbi_set_dust_species(rossbi_grid* g, const double* stokes_factor, int n);

/* The vertical sheared damped boundary (rossbi_vertical_damping_params).
 * Inside |z| > z_edge the five conservative gas departures relax towards the
 * equilibrium, dE'/dt = -E' R(z) / tau(r), R the parabola that is 1 at
 * |z| = z_max and 0, with zero slope, at z_edge (rates tabulated at cell
 * centres); the rate adds to the radial zones' and, like it, is a term of G
 * (both RK stages and rossbi_adjoint_step).  Dust is not damped.  p == NULL
 * switches it off (the default); otherwise 0 <= z_edge < z_max and
 * period_factor > 0.  Cylindrical grids with a disc equilibrium, symmetric
 * about z = 0, only.  Synchronises the stream.
 * Errors: ROSSBI_ERR_ARG, ROSSBI_ERR_OOM, ROSSBI_ERR_CUDA. */
rossbi_status rossbi_set_vertical_damping(rossbi_grid* g, const rossbi_vertical_damping_params* p);

/* The disc moments (A_disc, B_disc) of Sect. 2.10 of a state, without the
 * constant X_ref: the sums over cells of V (rho - rho_0 + rho_d) r cos(theta)
 * / R^3 and ... r sin(theta) / R^3 at the cell centres, in FP64 and in a
 * fixed order, exactly as the stage kernels take them.  They measure how far
 * the disc's mass is off centre; the indirect term need not be on.
 *   state : nfields device pointers of the grid's precision form.
 *   ab    : host array of 2 doubles receiving (A_disc, B_disc).
 * Cylindrical grids with an equilibrium set only.  Allocates the indirect
 * tables on first use; synchronises the stream.
 * Errors: ROSSBI_ERR_ARG, ROSSBI_ERR_OOM, ROSSBI_ERR_CUDA. */
rossbi_status rossbi_indirect_moments(rossbi_grid* g, const void* const* state, double* ab);

/* Copies the equilibrium conservative gas state at cell centres to host
 * memory: host_out[f*nz*nr + k*nr + i], f = 0..4 (App. B order). */
rossbi_status rossbi_get_equilibrium(rossbi_grid* g, double* host_out);

/* Global CFL time step of Sect. 2.5, Eq. (cfl condition):
 * dt = min over cells of cfl * V / ((|v| + c_s) max face area), with the
 * frame-relative speed; a dust cell adds cfl * V / (|v_d| max face area).
 * state: nfields device pointers of the grid's precision form.
 * Writes *dt_out (host) and also leaves dt on the device for a following
 * rossbi_step(..., dt = 0, ...).  Synchronises the stream. */
rossbi_status rossbi_cfl_dt(rossbi_grid* g, const void* const* state, double* dt_out);

/* One midpoint RK2 step (Sect. 2.5) of length dt, in place:
 *   E* = E^n + (dt/2) (G(E^n) - R0)/V, then drag over dt/2,
 *   E^{n+1} = E^n + dt (G(E*) - R0)/V, then drag over dt,
 * where G = S V - sum_faces A F.n (Sect. 2.2) and the drag is the closed-form
 * semi-implicit relaxation of the gas-dust relative velocity.  In the
 * perturbation forms G - R0 is evaluated directly as G(E0 + E') - G(E0).
 *   state   : nfields caller-owned device pointers, read and overwritten.
 *   scratch : nfields device pointers of the same type and size for E*, or
 *             NULL to use a buffer the library allocates on first use; none
 *             may be one of the state pointers (ROSSBI_ERR_ARG).
 *   dt      : > 0 uses this step; 0 uses the device-resident step left by the
 *             previous rossbi_step or rossbi_cfl_dt (no host round trip).
 *   dust    : drag parameters; required when n_dust = 1, ignored otherwise.
 *   next_dt : if not NULL, receives the CFL step of E^{n+1} (fused into the
 *             second stage) and the call synchronises and reports the status
 *             word.  If NULL the call is asynchronous and the next CFL step
 *             stays on the device.
 * Errors: ROSSBI_ERR_ARG, ROSSBI_ERR_OOM, ROSSBI_ERR_CUDA, and after a
 * synchronising call ROSSBI_ERR_NONPHYSICAL / ROSSBI_ERR_RIEMANN. */
rossbi_status rossbi_step(rossbi_grid* g, void* const* state, void* const* scratch, double dt,
                          const rossbi_dust_params* dust, double* next_dt);

/* Same step on HOST buffers: copies the state (nfields host pointers) to
 * device buffers owned by the library, steps, and copies it back; the call
 * synchronises.  For callers whose state lives in host memory. */
rossbi_status rossbi_step_host(rossbi_grid* g, void* const* host_state, double dt, const rossbi_dust_params* dust,
                               double* next_dt);

/* rossbi_step without any device allocation.  The paper has no counterpart:
 * this entry point serves callers that cannot call cudaMalloc while stepping,
 * for example host codes that give all device memory to their own pool
 * allocator at start-up, or loops that cannot accept the device-wide
 * synchronisation a cudaMalloc or cudaFree may cause.
 * Same arguments and result as rossbi_step with scratch == NULL, except that
 * the intermediate state E* and the reduction partials live in a fixed
 * 64 MiB (67,108,864-byte) array inside the library, allocated with the
 * library image on every GPU that loads it and held until the process exits.
 * Limit: nfields * (cells * element size, rounded up to 256 bytes) plus
 * (nfields + 1) * 8 bytes per 504-cell tile must fit in 64 MiB (for example
 * 9 fields in FP32 up to ~1.8 M cells, 5 fields in FP64 up to ~1.6 M cells);
 * larger grids get ROSSBI_ERR_ARG and nothing runs.
 * The grid's device (the one current at rossbi_init_grid) must be current
 * at every call, or the call returns ROSSBI_ERR_ARG: the array has one copy
 * per device.  The first call on a device looks the array's device address
 * up (with that device current); make that first call before any stream
 * capture.  Optional terms switched on with rossbi_set_indirect or
 * rossbi_set_damping act exactly as in rossbi_step (their tables are
 * allocated by those calls, not here).  Every
 * call shares the array and it keeps the last call's contents; nothing in it
 * needs to start at zero.  Calls that overlap on the GPU (other streams,
 * grids or host threads) race on the array: serialise them. */
rossbi_status rossbi_step_noalloc(rossbi_grid* g, void* const* state, double dt, const rossbi_dust_params* dust,
                                  double* next_dt);

/* Discrete adjoint of one rossbi_step at a fixed step length dt (FP64 form
 * only).  The paper has no adjoint; this is the exact transpose of the
 * linearised step map E^n -> E^{n+1} of Sect. 2.5: every branch (MinMod
 * limiter, Riemann wave pattern and sampling of Sect. 2.6, dust upwinding,
 * positivity fallback) is held where the forward values put it, and the star
 * pressure's derivative is dp* = -(df_L + df_R + du_R - du_L) / (f_L' + f_R')
 * at the converged p* (implicit function theorem).  The CFL choice of dt is
 * not differentiated: dt is an input.
 *   state_n : nfields device pointers holding E^n (read only); the call
 *             recomputes E*, the pre-drag stage states and E^{n+1} from it.
 *   dt      : > 0, the step that took E^n to E^{n+1}.
 *   dust    : drag parameters (required when n_dust = 1).
 *   lam_np1 : nfields device pointers, the cotangent of E^{n+1} (FP64).
 *   lam_n   : nfields device pointers receiving the cotangent of E^n; may
 *             be the same buffers as lam_np1 (in place).  Neither cotangent
 *             may share a pointer with state_n (ROSSBI_ERR_ARG).
 *   dparam  : if not NULL, receives += lam_np1 . dE^{n+1}/dSt (the Stokes
 *             number of dust), and the call synchronises and reports the
 *             status word.  The same value is always added to a device-side
 *             running total (rossbi_adjoint_dstokes), so callers can leave
 *             dparam NULL and keep the call asynchronous.
 * The library allocates five FP64 states of scratch on the first call.
 * Errors: ROSSBI_ERR_ARG, ROSSBI_ERR_UNSUPPORTED (perturbation forms, more
 * than one dust species),
 * ROSSBI_ERR_OOM, ROSSBI_ERR_CUDA, and after a synchronising call
 * ROSSBI_ERR_NONPHYSICAL / ROSSBI_ERR_RIEMANN. */
rossbi_status rossbi_adjoint_step(rossbi_grid* g, const void* const* state_n, double dt,
                                  const rossbi_dust_params* dust, const void* const* lam_np1, void* const* lam_n,
                                  double* dparam);

/* Running total of the d/dSt terms of every rossbi_adjoint_step on this grid;
 * reset != 0 sets it back to zero after reading.  Synchronises the stream. */
rossbi_status rossbi_adjoint_dstokes(rossbi_grid* g, double* total, int reset);

/* FP64 conservation sums sum_cells V * E_f of the FULL conservative fields
 * (E0 + E' in the perturbation forms), in a fixed reduction order (so the
 * result is deterministic).  sums: host array of nfields doubles.
 * Synchronises the stream. */
rossbi_status rossbi_conservation_sums(rossbi_grid* g, const void* const* state, double* sums);

/* Perturbation forms: number of Riemann faces solved so far by the FP64
 * full-state fallback (vacuum generation, strong rarefaction or slow Newton
 * convergence of the perturbation solver).  Synchronises the stream. */
rossbi_status rossbi_fallback_count(rossbi_grid* g, unsigned long long* count);

/* Waits for the stream, then returns and clears the device status word. */
rossbi_status rossbi_take_status(rossbi_grid* g);

/* Measurement: when enabled, every stage-kernel launch of rossbi_step is
 * bracketed by CUDA events recorded on the grid's stream.  rossbi_profile_read
 * synchronises the stream, returns the summed device time (ms) and the number
 * of stage launches since the last read, and resets both. */
rossbi_status rossbi_profile_enable(rossbi_grid* g, int enable);
rossbi_status rossbi_profile_read(rossbi_grid* g, double* stage_ms, int* stage_launches);

/* Measurement: the device's fused multiply-add throughput in FLOP/s (2 per
 * FMA), FP32 (fp64 = 0) or FP64 (fp64 != 0), timed with CUDA events on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream) over a kernel
 * of eight independent FMA chains per thread on 8 blocks of 256 threads per
 * SM, after one warm-up launch: the ALU roof against which the stage
 * kernels' arithmetic is reported.  Takes ~0.1 s; synchronises the stream.
 * Errors: ROSSBI_ERR_ARG (flops_per_s == NULL), ROSSBI_ERR_OOM,
 * ROSSBI_ERR_CUDA. */
rossbi_status rossbi_measure_fma_peak(int fp64, void* cuda_stream, double* flops_per_s);

/* Number of conservative fields (5 + 4 n_dust) and the precision form. */
int rossbi_nfields(const rossbi_grid* g);
int rossbi_precision(const rossbi_grid* g);

/* Frees every library-owned resource of the grid (not the caller's state). */
void rossbi_destroy(rossbi_grid* g);

/* Static, human-readable name of a status code. */
const char* rossbi_status_string(rossbi_status s);

#ifdef __cplusplus
}
#endif

#endif /* ROSSBI_H */
