/*
 * lbm.h -- C ABI of the GB300 (sm_103a) axisymmetric Allen-Cahn phase-field
 * multiple-relaxation-time lattice Boltzmann library (libaxilbm.so).
 *
 * The method is that of Liang et al., "Axisymmetric lattice Boltzmann model for
 * multiphase flows with large density ratio" (arXiv 1810.09299): a phase-field
 * LBE for the conservative Allen-Cahn equation (Sec. 2.2, Eq. 9-23) coupled to a
 * pressure-based hydrodynamic LBE (Sec. 2.3, Eq. 24-37) on a D2Q9 (z, r)
 * lattice, with the isotropic stencils of Eq. 39-40 for the only non-local
 * field phi, the axis-symmetry boundary at r = 0 and bounce-back walls.
 *
 * Conventions used by every entry point
 *   - Lattice node (k, j): k = 0..nz-1 along z, j = 0..nr-1 along r.  The first
 *     lattice line sits at r = 0.5 (Sec. 2.3): r_j = j + 0.5, z_k = k + 0.5.
 *   - Host arrays are FP64, row-major [z][r] (r fastest), in every precision.
 *   - Return value: LBM_OK (0) or a negative lbm_status.  Errors are sticky: once
 *     a call on a handle fails with LBM_ERR_CUDA or LBM_ERR_NONFINITE, every later
 *     call on that handle returns the same code until lbm_destroy.
 *   - The library owns all device memory of a handle.  It is allocated
 *     stream-ordered on the stream given at creation and freed by lbm_destroy.
 *     Host pointers passed in are borrowed for the duration of the call only.
 *   - All device work is enqueued on the handle's stream.  Calls that return host
 *     data (lbm_get_fields, lbm_diagnostics, lbm_get_state, lbm_checkpoint_save)
 *     synchronise that stream; lbm_step does not.
 *   - A handle is not thread-safe: one host thread at a time.
 */
#ifndef AXILBM_LBM_H
#define AXILBM_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sim lbm_handle;   /* one case, or a batch of cases */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = -1,  /* a parameter is out of range or a pointer is NULL */
    LBM_ERR_CUDA = -2,         /* a CUDA runtime call or a kernel launch failed */
    LBM_ERR_NONFINITE = -3,    /* a NaN or Inf appeared in phi, u or p */
    LBM_ERR_TIMEOUT = -4,      /* a bounded device wait gave up (see lbm_step) */
    LBM_ERR_OOM = -5,          /* device allocation failed */
    LBM_ERR_STATE = -6         /* call out of order (e.g. lbm_step before lbm_init_phase) */
} lbm_status;

/* Storage and arithmetic precision of a handle.
 *   LBM_FP64      populations and arithmetic in FP64.
 *   LBM_FP32      populations f_1..8 and g_0..8 in FP32, arithmetic in FP32
 *                 (reciprocals, divisions and square roots by the hardware
 *                 approximations, a few ulp, subnormal operands and results
 *                 flushed to zero; the same in the two 16-bit forms).
 *                 f_0 is stored as a pair of FP32 numbers holding the node's
 *                 mass ledger: (sum of its incoming populations) minus (its
 *                 stored outgoing f_1..8), accumulated with error-free FP32
 *                 additions, so the sum of all populations (the conserved sum
 *                 of r phi, Eq. 16) changes only by round-off of about 2^-48.
 *   LBM_MIX_FP16  populations f_1..8 and g_0..8 stored as FP16 deviations
 *                 f_i / S_i - 1/2 and 256 g_i / S_i, S_i = w_i r of the
 *                 storing node rounded up to 2 significant bits in the ratios
 *                 of the weights, the f deviation on a 2^-14 grid; arithmetic
 *                 in FP32; reductions in FP64.  Every stored f_i then decodes
 *                 exactly, to a multiple of a per-column grid, so f_0, one
 *                 FP32 number, holds the node's mass ledger in exact FP32
 *                 arithmetic: the step conserves the sum of all populations
 *                 exactly.  nr <= 65536.
 *   LBM_MIX_BF16  populations stored as bfloat16 deviations f_i / (w_i r) - 1/2
 *                 and g_i / (w_i r) on the full FP32 scale w_i r; f_0 is the
 *                 double-float ledger of LBM_FP32 (round-off of about 2^-48).
 *                 nr <= 65536.  bfloat16 keeps 8 significant bits: slowly
 *                 moving interfaces can pin where the per-step change is below
 *                 that resolution. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_MIX_FP16 = 2, LBM_MIX_BF16 = 3 } lbm_precision;

/* Coupling of the pressure p and the radial velocity u_r (Eq. 32 uses p, Eq. 33
 * computes p from u).  LBM_P_EXACT solves both together at each node (the pair is
 * a quadratic in p; the root continuous with the linear solution is taken).
 * LBM_P_LAGGED uses p^{n-1} in Eq. 32 and Eq. 30. */
typedef enum { LBM_P_EXACT = 0, LBM_P_LAGGED = 1 } lbm_p_coupling;

/* Moment basis of both collisions (Eq. 19 and Eq. 24).
 *   LBM_MRT_ORTHOGONAL  the paper's orthogonal moments, M of Sec. 2.2.
 *   LBM_MRT_RAW         the non-orthogonal raw moments 1, c_z, c_r, c_z^2 + c_r^2,
 *                       c_z^2 - c_r^2, c_z c_r, c_z^2 c_r, c_z c_r^2, c_z^2 c_r^2: the
 *                       extension the paper's summary names (Sec. 4).  sf and sg
 *                       then give the rates of these nine moments, and s_p of
 *                       Eq. 33 becomes 3 / (2 s_3) - 1 / (2 s_8) - 1/2 (Appendix C
 *                       redone in this basis).  The paper's rate choice reads
 *                       sf = (1, s, s, 1, 1, 1, s, s, 1), for which the f-collision
 *                       is the paper's own, and sg = 1 except s_3 = s_4 = s_5 =
 *                       1/tau_g.  With this choice (rates derived as in the
 *                       paper) the step runs kernels specialised for it, as for
 *                       the paper's own pattern; other rates run the general
 *                       kernels. */
typedef enum { LBM_MRT_ORTHOGONAL = 0, LBM_MRT_RAW = 1 } lbm_collision;

/* Parameters of one case.
 *   nr, nz       lattice size (nr >= 2, nz >= 2).
 *   z_periodic   1: periodic in z; 0: halfway bounce-back walls at z = 0 and z = nz.
 *                The wall at r = nr is always a halfway bounce-back wall and the
 *                axis r = 0 always a symmetry line (Sec. 2.3).
 *   rho_l, rho_g liquid (phi = 1) and gas (phi = 0) densities, Eq. 17 (> 0).
 *   nu_l, nu_g   kinematic viscosities, Eq. 35 (> 0).
 *   sigma, W     surface tension and interface width: k = 1.5 sigma W and
 *                beta = 12 sigma / W in Eq. 4 (sigma >= 0, W > 0).
 *   mobility     M of Eq. 1 and Eq. 11; tau_f = M / cs2 + 1/2 (Eq. 18) (> 0).
 *   grav_z       z component of gravity; body force G = ((rho - rho_l) grav_z, 0).
 *   sf[9], sg[9] diagonal MRT rates of Eq. 13 and Eq. 28, each in [0, 2).  A
 *                negative entry is derived: sf -> 1/tau_f, sg -> 1/tau_g(x) with
 *                nu(x) = cs2 (tau_g - 1/2) at every node (Eq. 34).
 *   n_eps        interface normal n = grad phi / (|grad phi| + n_eps).
 *   precision    lbm_precision; p_coupling lbm_p_coupling; collision
 *                lbm_collision. */
typedef struct {
    int32_t nr, nz, z_periodic;
    int32_t precision;
    int32_t p_coupling;
    int32_t collision;
    double rho_l, rho_g, nu_l, nu_g, sigma, W, mobility, grav_z;
    double sf[9], sg[9];
    double n_eps;
} lbm_params;

/* Diagnostics record: the quantities the paper reads off its runs -- the
 * conserved sum of r phi (Eq. 16), the pressure jump of Laplace's law and the
 * spurious-velocity maximum of the static drop (Sec. 3.1), the axis half-length
 * whose oscillation gives the frequency of Sec. 3.2 (Eq. 43-45) -- all FP64,
 * computed on the device in a fixed order (deterministic): each of a fixed set
 * of blocks sums its nodes plainly and then pairwise, and the block results
 * are combined with compensated (Neumaier) sums.  A node whose phi, u_z, u_r
 * or p is not finite is left out of every sum and extremum and counted in
 * nonfinite.
 *   mass               sum over nodes of r phi (equal to the sum of all f_i).
 *   kinetic            sum of 0.5 r rho |u|^2.
 *   z_centroid         sum r z phi / sum r phi.
 *   dp                 <p> over phi > 0.99 minus <p> over phi < 0.01 (r-weighted).
 *   umax               max |u|.
 *   axis_half_length   half the length of the phi > 1/2 set on the axis row j = 0,
 *                      from linear interpolation of the crossings.
 *   radial_half_length first phi = 1/2 crossing along r on the row nearest z_centroid.
 *   nonfinite          number of nodes with a non-finite phi, u or p. */
typedef struct {
    double step, mass, kinetic, z_centroid, dp, umax, phi_min, phi_max;
    double axis_half_length, radial_half_length, nonfinite;
} lbm_diag;

/* Initial phase-field shapes for lbm_init_phase (coordinates z = k+0.5, r = j+0.5).
 *   FLAT      args {z_i, W, axis}: phi = 1/2 + 1/2 tanh(2 (z_i - x) / W), x = z (axis 0) or r.
 *   SPHERE    args {z_c, R, W}: drop of Eq. 41, phi = 1/2 + 1/2 tanh(2 (R - d) / W).
 *   ELLIPSOID args {z_c, R_z, R_r, W}: Eq. 46 with R_e = (R_r^2 R_z)^(1/3).
 *   P2        args {z_c, R0, eps, W}: drop of radius R0 (1 + eps P2(cos theta)).
 *   THREAD    args {R, amp, lambda, theta, W}: Eq. 47 with d = amp cos(2 pi z / lambda + theta).
 *   BUBBLE    args {z_c, R, W}: 1 - SPHERE.
 *   HOST_ARRAY host_phi [nz][nr] is copied to the device. */
typedef enum {
    LBM_SHAPE_FLAT = 0, LBM_SHAPE_SPHERE = 1, LBM_SHAPE_ELLIPSOID = 2, LBM_SHAPE_P2 = 3,
    LBM_SHAPE_THREAD = 4, LBM_SHAPE_BUBBLE = 5, LBM_SHAPE_HOST_ARRAY = 6
} lbm_shape;

/* Field selection bits for lbm_get_fields; fields are written in bit order. */
enum { LBM_FIELD_PHI = 1, LBM_FIELD_RHO = 2, LBM_FIELD_UZ = 4, LBM_FIELD_UR = 8, LBM_FIELD_P = 16 };

/* Create a single-case handle.  stream: a cudaStream_t (NULL = default stream).
 * Validates the parameters (LBM_ERR_INVALID_ARG; among them nz * pitch < 2^31
 * with pitch = nr rounded up to 32), allocates the device state (LBM_ERR_OOM)
 * and selects the current CUDA device.  *out is set on success. */
int lbm_create(const lbm_params* prm, void* stream, lbm_handle** out);
/* The parameters are those of the paper's model: the densities of Eq. 17,
 * the viscosities of Eq. 35 that give tau_g through Eq. 34, sigma and W that
 * give beta and k of Eq. 4, the mobility that gives tau_f through Eq. 18, and
 * the diagonal rates of Eq. 13 (phase field) and Eq. 28 (hydrodynamics). */

/* Create a batch of ncases independent cases (ncases >= 1) that advance together:
 * each lbm_step launch covers the tiles of every case (Sec. 3's test problems run
 * side by side).  All cases must share one precision. */
int lbm_batch_create(const lbm_params* cases, int32_t ncases, void* stream, lbm_handle** out);

/* Number of cases of a handle (1 for lbm_create). */
int32_t lbm_num_cases(const lbm_handle* h);

/* Initial condition of case `icase` (Sec. 3, the paper is silent beyond phi):
 * phi0 from the shape, u = 0, p = 0, f = f^eq(phi0, u = 0) (Eq. 11), g = 0
 * (= g^eq at p = 0, u = 0, Eq. 25), chi^{-1} = (0, M phi0) so that the first
 * time derivative of Eq. 38 is zero, p^{-1} = 0.  Resets the step counter.
 * nargs must match the shape (see lbm_shape); host_phi is used only for
 * LBM_SHAPE_HOST_ARRAY.  lbm_init_phase initialises case 0. */
int lbm_init_phase(lbm_handle* h, int32_t shape, const double* shape_args, int32_t nargs,
                   const double* host_phi);
int lbm_case_init_phase(lbm_handle* h, int32_t icase, int32_t shape, const double* shape_args,
                        int32_t nargs, const double* host_phi);

/* The same initial condition for every case of the handle at once, from host
 * arrays: host_phi holds each case's phi0 ([nz][nr] doubles) one after the
 * other, in case order (sum over cases of nz * nr doubles).  One host-to-device
 * copy and one synchronisation for the whole batch, instead of one per case.
 * The first call allocates a device staging array of that size, kept until
 * lbm_destroy.  Resets every step counter.  Synchronises. */
int lbm_init_phase_all(lbm_handle* h, const double* host_phi);

/* Advance every case by nsteps time steps (nsteps >= 0).  One step is
 * Eq. 16 (phi) -> Eq. 39-40 (stencils) -> Eq. 4, 17, 35 -> Eq. 32-33 (u, p) ->
 * Eq. 30 (force) -> Eq. 19-23 (phase-field collision) -> Eq. 24-29, 36-37
 * (hydrodynamic collision) -> Eq. 20 (streaming with axis reflection and
 * bounce-back).  Asynchronous on the handle's stream; repeated steps are
 * replayed from a captured CUDA graph.  Returns launch errors immediately and
 * earlier sticky errors.  The launch shapes that stage tiles through shared
 * memory with TMA copies (lbm_set_variant) wait on them with a bounded number
 * of polls; a wait that gives up is reported later as LBM_ERR_TIMEOUT.  A copy
 * of that CTA may then still have been in flight when it left, so after
 * LBM_ERR_TIMEOUT treat the CUDA context as suspect: destroy the handle and
 * create a new one (in a new process if the error returns). */
int lbm_step(lbm_handle* h, int64_t nsteps);

/* Copy macroscopic fields of case 0 / case icase to the host:
 * host_out holds popcount(mask) arrays of [nz][nr] doubles, in bit order of
 * LBM_FIELD_*: phi = sum f_i / r (Eq. 16), rho (Eq. 17), u (Eq. 31-32) and
 * p (Eq. 33, solved with u_r as lbm_p_coupling says), recomputed from the
 * current populations exactly as the next step computes them.  Synchronises. */
int lbm_get_fields(lbm_handle* h, int32_t mask, double* host_out);
int lbm_case_get_fields(lbm_handle* h, int32_t icase, int32_t mask, double* host_out);

/* Diagnostics of case 0 / case icase (see lbm_diag: the quantities of
 * Sec. 3.1-3.2).  Synchronises.  Returns LBM_ERR_NONFINITE (and fills *out)
 * if any phi, u or p is not finite. */
int lbm_diagnostics(lbm_handle* h, lbm_diag* out);
int lbm_case_diagnostics(lbm_handle* h, int32_t icase, lbm_diag* out);

/* One liquid drop on the axis (see lbm_case_axis_drops). */
typedef struct {
    double z_start, z_end;  /* phi = 1/2 crossings on the axis; z_end < z_start when it wraps */
    double volume;          /* 2 pi sum r phi over the rows of the drop */
    double radius;          /* radius of the sphere of that volume */
} lbm_drop;
#define LBM_MAX_AXIS_DROPS 64

/* The drops along the axis of case icase: the liquid bodies that a breaking
 * liquid thread forms (Sec. 3.3), from which its breakup time and the sizes
 * of its main and satellite drops are read.  Each maximal run of nodes of the
 * axis row (j = 0) with phi > 1/2 is one drop (its ends: the interpolated
 * phi = 1/2 crossings, or a z wall plane).  Every row of the case belongs to
 * one drop: each gas gap on the axis is split at its row of least
 * sum_j r_j phi (the first such row), and a drop's volume is 2 pi sum r phi over
 * its rows.  In a z-periodic case the rows wrap around; with phi > 1/2 along
 * the whole axis the case holds one unbroken body (z_start = 0, z_end = nz).
 * A thread has broken once the least phi of the axis row falls below 1/2.
 *   max_drops   0 .. LBM_MAX_AXIS_DROPS: records to write to drops[], in z
 *               order from the scan start (z = 0, or in a periodic case the
 *               first gas gap after z = 0).
 *   n_drops     number of drops found (may exceed max_drops).
 *   axis_min    NULL, or 2 doubles: the least phi of the axis row and its z.
 * Computed on the device in FP64 from the fields of lbm_get_fields.
 * Synchronises.  LBM_ERR_INVALID_ARG for a bad case, count or pointer,
 * LBM_ERR_STATE before the case's initial condition. */
int lbm_case_axis_drops(lbm_handle* h, int32_t icase, int32_t max_drops, lbm_drop* drops, int32_t* n_drops,
                        double* axis_min);

/* Pipelined diagnostics: the record of lbm_case_diagnostics (the quantities
 * Sec. 3.1-3.3 read off the runs), enqueued on the handle's stream without
 * waiting, so that a loop reading one record per step keeps the GPU busy:
 * enqueue step n and its record, enqueue step n+1, then wait for record n.
 *   host_out  the lbm_diag the record is copied into when the stream gets
 *             there.  Unlike other host pointers it is kept beyond the call:
 *             it must stay valid until lbm_diagnostics_wait on its slot
 *             returns.  Use page-locked (pinned) memory; with pageable memory
 *             the copy, and with it this call, completes before returning.
 *   slot      0 .. LBM_DIAG_SLOTS - 1, names the record for the wait; an
 *             enqueue on a slot replaces the slot's previous record (wait for
 *             that one first).
 * Returns LBM_ERR_INVALID_ARG for a bad case or slot or a NULL host_out,
 * LBM_ERR_STATE if the case has no initial condition.  Does not synchronise. */
#define LBM_DIAG_SLOTS 4
int lbm_case_diagnostics_enqueue(lbm_handle* h, int32_t icase, lbm_diag* host_out, int32_t slot);

/* Wait until the record enqueued on `slot` is in its host_out.  Returns
 * LBM_ERR_TIMEOUT if a bounded device wait gave up before it, LBM_ERR_NONFINITE
 * if the record counts non-finite values (both sticky, as for
 * lbm_case_diagnostics), LBM_ERR_STATE if nothing is pending on the slot. */
int lbm_diagnostics_wait(lbm_handle* h, int32_t slot);

/* Populations of case icase as FP64 host arrays f[9][nz][nr], g[9][nz][nr] and the
 * time-level state aux[3][nz][nr] = (chi_z^{n-1}, chi_r^{n-1}, p^{n-1}); any pointer
 * may be NULL.  lbm_set_state writes them (encoding to the storage precision).
 * Synchronises. */
int lbm_get_state(lbm_handle* h, int32_t icase, double* f, double* g, double* aux);
int lbm_set_state(lbm_handle* h, int32_t icase, const double* f, const double* g, const double* aux);

/* Checkpoint / resume of the whole handle in its native storage precision.
 * lbm_checkpoint_size returns the byte size of the image; save/load copy it
 * to / from host memory of at least that size.  Resuming from a checkpoint is
 * bit-identical to running straight through.  Synchronises. */
int64_t lbm_checkpoint_size(const lbm_handle* h);
int lbm_checkpoint_save(lbm_handle* h, void* host_buf);
int lbm_checkpoint_load(lbm_handle* h, const void* host_buf);

/* Time a few launch shapes of the step kernel on the current state (which is
 * saved and restored, so the simulation does not advance) and keep the fastest.
 * Candidates are timed in index order; a later one must be at least 1 % faster
 * than the best so far to replace it, so near ties keep the earlier shape.
 * reps >= 1 timed steps per candidate.  Writes the chosen variant index to
 * *chosen (may be NULL).  Synchronises. */
int lbm_autotune(lbm_handle* h, int32_t reps, int32_t* chosen);

/* Select a step-kernel launch variant explicitly (0 .. lbm_num_variants()-1).
 * Every variant computes bit-identical results; they differ in tile height
 * (rows along z of the 32-column tile), in nodes per thread and in staging:
 *   0, 1, 2  one node per thread, tiles of 8, 16, 4 rows;
 *   3, 4     one node per thread, tiles of 8, 16 rows staged in shared memory
 *            by TMA copies (persistent, pipelined; needs the tensor maps);
 *   5, 6     two nodes of a column per thread, tiles of 16 rows; 6 keeps the
 *            second node's stored inputs in shared memory while the first is
 *            updated (FP64 handles run the one-node kernel of 16 rows)
 *   7        LBM_MIX_FP16: two nodes of a column per thread whose macroscopic
 *            step and collisions run together in packed FP32x2 lanes; other
 *            precisions run variant 5 here. */
int lbm_set_variant(lbm_handle* h, int32_t variant);
int32_t lbm_num_variants(void);

/* Number of step-kernel launches this handle has issued (one per step). */
int64_t lbm_kernel_launches(const lbm_handle* h);

/* Allocation-free diagnostics reduction.  The paper has no counterpart: this
 * is a service for callers that cannot allocate device memory at the moment
 * they need the numbers (their device memory is held by their own pool, or
 * they run a monitoring loop that must not pay for an allocation).
 *   d_fields  device pointer, FP64 [5][nz][nr]: phi, rho, u_z, u_r, p (the
 *             layout lbm_get_fields uses with mask 31), read only.
 *   d_out     device pointer to 11 doubles, written with the lbm_diag record
 *             (same definitions, same kernels and summation order as
 *             lbm_diagnostics); step is copied into the first entry.
 *   stream    cudaStream_t the work is enqueued on (NULL: default stream);
 *             the call returns without synchronising.
 * Nothing is allocated: the only scratch is a fixed 43,776-byte static device
 * array of the library, held on every GPU that loads it until the process
 * exits.  Requires nz, nr >= 1 and nz * nr <= 2^31 - 1, else
 * LBM_ERR_INVALID_ARG.  The first call on a device looks up that array's
 * device address on the current device; make that first call before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or anything else that replaces the device's primary
 * context) it is stale, so do not call this entry point again in that
 * process.  All calls share the array (its contents are fully rewritten by
 * each call), so calls that overlap on the GPU, e.g. on two streams, race. */
int lbm_diag_reduce_noalloc(const double* d_fields, int32_t nz, int32_t nr, int32_t z_periodic, double step,
                            double* d_out, void* stream);

/* Self-test of the library's bounded device waits (no paper counterpart):
 * launches a kernel whose mbarrier phase can never complete and whose wait
 * therefore gives up after `tries` polls, writing 1 to the device int
 * *device_status_word (device memory, caller-owned, should hold 0 on entry).
 * Returns LBM_ERR_TIMEOUT when the wait gave up as designed, LBM_OK if it did
 * not, LBM_ERR_INVALID_ARG for tries < 1 or a NULL pointer.  Synchronises
 * `stream`.  The context stays usable: the kernel leaves no work in flight. */
int lbm_selftest_bounded_wait(int32_t tries, void* stream, int32_t* device_status_word);

/* Measured throughput of the GPU's FP64 pipe (no paper counterpart: the
 * denominator of the FP64 step's arithmetic roofline, whose step is bound by
 * that pipe rather than by memory).  Launches 4 blocks of 256 threads per SM,
 * each thread running 8 independent chains of `iters` dependent FP64 fused
 * multiply-adds, after one untimed warm-up launch, and writes the FMA count
 * over the CUDA-event time of the timed launch to *fma_per_second.  Allocates
 * and frees a small device buffer; synchronises `stream`.  LBM_ERR_INVALID_ARG
 * for iters < 1 or a NULL pointer. */
int lbm_measure_fp64_rate(int32_t iters, void* stream, double* fma_per_second);

/* Release every resource of the handle (NULL is ignored).  No paper
 * counterpart: resource management only. */
int lbm_destroy(lbm_handle* h);

/* Static description of a status code. */
const char* lbm_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif
