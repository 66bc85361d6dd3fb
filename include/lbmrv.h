/*
 * lbmrv — lattice Boltzmann schemes with relative velocities on one GB300 (sm_103a).
 *
 * C ABI of the library. The method is that of F. Dubois, T. Fevrier and B. Graille,
 * "Lattice Boltzmann schemes with relative velocities" (arXiv:1312.3297):
 *   - Section 1.1: a time step is a local relaxation in moment space followed by the
 *     exact transport f_j(x, t+dt) = f*_j(x - v_j dt, t) (relation (transport));
 *   - Section 1.2: the moments are taken in a frame moving at a relative velocity u~,
 *     m(u~) = M(u~) f with M(u~)_kj = P_k(v_j - u~) (relations (MatMu), (ftomu)),
 *     relaxed diagonally towards m_eq(u~) = M(u~) f_eq (relation (relaxationu)),
 *     and mapped back f* = M(u~)^{-1} m*;
 *   - Section 1.3: for D2Q9 with the orthogonal moments of relation (mom),
 *     M(u~) = T(u~) M(0) with the lower block-triangular shifting matrix T(u~)
 *     (relation (matTu), Appendix A) and T(u~)^{-1} = T(-u~) (morphism proposition).
 * u~ = 0 is d'Humieres' MRT scheme; u~ = q/rho is the cascaded-like choice; u~ may also
 * be a prescribed field u~(x, t).
 *
 * Conventions shared by every entry point:
 *   - Return value: LBMRV_OK (0) or a negative LBMRV_E_* status. Nothing is thrown
 *     across the ABI. lbmrv_last_error() gives a one-line message for the last failure.
 *   - Pointers named *_dev are device pointers (CUDA global memory of the handle's
 *     device); pointers named *_host are host pointers. Caller-owned buffers are never
 *     freed or retained by the library beyond the call, except the buffers passed to
 *     lbmrv_create and lbmrv_set_utilde, which must outlive the handle (or the next
 *     lbmrv_set_utilde call).
 *   - Work is enqueued on the handle's CUDA stream and returns without synchronising,
 *     except the calls documented as synchronous (they return host values). Step kernels
 *     are launched with programmatic dependent launch: one may be scheduled while the work
 *     before it in the stream finishes, but it touches no memory until that work has
 *     completed, so stream order means what it always does.
 *   - Lattice layout: periodic D2Q9 (dims = {nx, ny, 1}) or D3Q19 (dims = {nx, ny, nz}),
 *     lattice units dx = 1 (so dt = 1/lambda, relation (lambda)). Node (x, y, z) has index
 *     i = (z*ny + y)*nx + x; n = nx*ny*nz. Population state: structure of arrays, q planes
 *     of n elements (q = 9 or 19); plane j holds velocity j, for D2Q9 in the order
 *     (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1) (times lambda) of Section
 *     1.3. Element i of plane j is at offset j*n + i. Velocity fields are d planes of n
 *     floats (d = 2 or 3).
 *   - Stored value: g_j = f_j - f_eq,j(rho_ref, U_ref), the deviation from the equilibrium
 *     of a reference state, in the storage type of the handle (FP32, FP16 or BF16,
 *     round-to-nearest-even). rho_ref is given at lbmrv_create (0 stores f itself when
 *     U_ref = 0). By default U_ref is chosen automatically by each lbmrv_init_equilibrium:
 *     the mean flow sum(rho u) / sum(rho) of its fields, which the periodic scheme
 *     conserves (relation (rhoq) summed over the lattice), so the stored deviations stay
 *     those of the perturbations around the mean flow and 16-bit rounding stays small.
 *     lbmrv_set_reference fixes U_ref instead (U_ref = 0 is the plain form
 *     g_j = f_j - w_j rho_ref, w = (4/9, 1/9 x4, 1/36 x4)); lbmrv_get_reference reports
 *     it. All arithmetic is FP32.
 *   - The state kept by the handle after k steps is the POST-relaxation state
 *     S_k = C_k(f(k)) at time k: one lbmrv_step pulls the neighbours' S_{k-1}
 *     (transport) and relaxes at time k. Moments (rho, q) of S_k equal those of f(k),
 *     since relaxation conserves them.
 */
#ifndef LBMRV_H
#define LBMRV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBMRV_VERSION 1

#if defined(__GNUC__)
#define LBMRV_API __attribute__((visibility("default")))
#else
#define LBMRV_API
#endif

/* Status codes. */
#define LBMRV_OK 0
#define LBMRV_E_INVAL (-1)       /* an argument is out of range or inconsistent */
#define LBMRV_E_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define LBMRV_E_NOMEM (-3)       /* device allocation failed, or a workspace is too small */
#define LBMRV_E_NONFINITE (-4)   /* a NaN or infinity was found in the state */
#define LBMRV_E_TIMEOUT (-5)     /* reserved: no entry point waits on the device */
#define LBMRV_E_UNSUPPORTED (-6) /* valid request that this library does not implement */

/* Lattices. D3Q19 uses 19 velocities (0,0,0); (+-1,0,0), (0,+-1,0), (0,0,+-1);
 * (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0); (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1);
 * (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1) (times lambda, in this order) and the 19
 * polynomials 1, X, Y, Z, X^2+Y^2+Z^2, X^2-Y^2, Y^2-Z^2, XY, XZ, YZ, XY^2, XZ^2, YX^2,
 * YZ^2, ZX^2, ZY^2, X^2Y^2, X^2Z^2, Y^2Z^2 (divided by lambda^degree from degree 2 on).
 * The paper prints no 3D basis; this one spans a space closed under differentiation, so
 * its shifting matrix is lower triangular with T(u~)^{-1} = T(-u~), as for D2Q9. */
#define LBMRV_D2Q9 0
#define LBMRV_D3Q19 1
/* D2Q9 with Geier's cascaded basis 1, X, Y, X^2+Y^2, X^2-Y^2, XY, XY^2, X^2Y, X^2Y^2
 * (relation (polgeier), divided by lambda^degree from degree 2 on; rates s[0..8] in this
 * order) and the product-form equilibrium whose moments in the fluid frame are those of
 * the Maxwellian, rho (1, 0, 0, 2 c^2, 0, 0, 0, 0, c^4), c^2 = lambda^2/3. With
 * LBMRV_UT_FLUID this is Geier's cascaded scheme (proposition of Section 1.3, Appendix B);
 * the other u~ modes apply as for LBMRV_D2Q9. No adjoint. */
#define LBMRV_D2Q9_CASCADED 2

/* Choice of the relative velocity u~ (Section 1.2, Introduction). */
#define LBMRV_UT_ZERO 0       /* u~ = 0: d'Humieres MRT */
#define LBMRV_UT_FLUID 1      /* u~ = q/rho of the node being relaxed */
#define LBMRV_UT_PRESCRIBED 2 /* u~(x, t) = A u~0(x) cos(2 pi t / P), see lbmrv_set_utilde */

/* Population storage types. */
#define LBMRV_FP32 0
#define LBMRV_FP16 1
#define LBMRV_BF16 2

typedef struct lbmrv_s* lbmrv_t;

/* Library version (LBMRV_VERSION). */
LBMRV_API int lbmrv_version(void);

/* Bytes of one population state (q * n * element size) for the given lattice, dims and
 * storage; -1 on invalid arguments. */
LBMRV_API int64_t lbmrv_state_bytes(int lattice, const int64_t dims[3], int storage);

/* Create a simulation handle on the current CUDA device.
 *   lattice  LBMRV_D2Q9, LBMRV_D2Q9_CASCADED or LBMRV_D3Q19.
 *   dims     {nx, ny, 1} or {nx, ny, nz}, all >= 1, n < 2^31.
 *   lambda   velocity scale lambda > 0 (relation (lambda)).
 *   s        q relaxation rates in basis order: for D2Q9 the moment order of relation
 *            (mom): rho, q_x, q_y, e, p_xx, p_xy, q_x(3rd), q_y(3rd), eps; for the other
 *            lattices the order of their bases above. The 1 + d conserved rates must be 0
 *            (Section 1.1); the others are finite. A rate outside (0, 2) is accepted with
 *            a warning in lbmrv_last_error (of the handle, and of NULL on this thread):
 *            that moment is then not damped (0 or 2) or amplified.
 *   umode    LBMRV_UT_* (prescribed mode: see lbmrv_set_utilde; default A = 0).
 *   storage  LBMRV_FP32 / LBMRV_FP16 / LBMRV_BF16.
 *   rho_ref  reference density of the stored deviation g = f - w rho_ref (0 stores f).
 *   stream   cudaStream_t to enqueue on (NULL: the legacy default stream).
 *   f_a_dev, f_b_dev
 *            two device buffers of lbmrv_state_bytes() each, 16-byte aligned, owned by
 *            the caller and used as the A-B pair of the pull step; or both NULL, and
 *            the library allocates (and later frees) them.
 * The handle also allocates a small reduction buffer (under 64 KB) and the nx-float table
 * sin(2 pi x / nx) of the analytic prescribed field.
 * Errors: LBMRV_E_INVAL, LBMRV_E_UNSUPPORTED, LBMRV_E_NOMEM, LBMRV_E_CUDA; *out is NULL. */
LBMRV_API int lbmrv_create(lbmrv_t* out, int lattice, const int64_t dims[3], double lambda,
                 const double* s, int umode, int storage, double rho_ref, void* stream,
                 void* f_a_dev, void* f_b_dev);

/* Release the handle and whatever it allocated. Synchronises its stream. NULL is a no-op. */
LBMRV_API int lbmrv_destroy(lbmrv_t h);

/* Message of the last failure (or rate warning) on h, or of the last failed (or warned)
 * lbmrv_create on this thread when h is NULL. Valid until the next call on h. */
LBMRV_API const char* lbmrv_last_error(lbmrv_t h);

/* Fixed reference state of the stored deviations: g = f - f_eq(rho_ref, u_ref), u_ref = d
 * doubles in physical units (NULL: zero, the plain form g = f - w rho_ref). It turns the
 * automatic choice off. It changes how the stored state is read and written, so call it
 * before lbmrv_init_equilibrium / lbmrv_set_state; an existing state is not converted.
 * Errors: LBMRV_E_INVAL (NULL handle, non-finite values). */
LBMRV_API int lbmrv_set_reference(lbmrv_t h, double rho_ref, const double* u_ref);

/* Automatic reference velocity (the default): from now on each lbmrv_init_equilibrium[_host]
 * sets U_ref to the mean flow sum(rho u) / sum(rho) of its fields (an FP64 reduction on the
 * device) before it builds the state, and rho_ref to the value given here. The mean flow
 * is an invariant of the periodic scheme (total mass and momentum are conserved), so it
 * remains the mean flow of every later state. lbmrv_set_state keeps the current
 * reference. Errors: LBMRV_E_INVAL (NULL handle, rho_ref not finite). */
LBMRV_API int lbmrv_set_reference_auto(lbmrv_t h, double rho_ref);

/* Current reference state: *rho_ref_out and u_ref_out[0..2] (physical units, unused
 * components 0); either pointer may be NULL. Returns 1 when the automatic choice is on,
 * 0 when the reference is fixed, LBMRV_E_INVAL for a NULL handle. */
LBMRV_API int lbmrv_get_reference(lbmrv_t h, double* rho_ref_out, double* u_ref_out);

/* Change the stream later work is enqueued on. */
LBMRV_API int lbmrv_set_stream(lbmrv_t h, void* stream);

/* Kernel variant of the fused step: 0 chooses automatically (the widest aligned pack that
 * divides nx, up to the width measured fastest for the lattice and storage), 1 forces one
 * node per thread (any lattice), 2/4/8 force that many consecutive nodes per thread with
 * vector loads (must divide nx; at most 4 for FP32, 8 for 16-bit storage; the state
 * buffers must be aligned to the pack). All variants compute the same scheme to rounding;
 * this exists for testing and tuning. Automatic widths: D2Q9 4 (FP32) or 8 (16-bit);
 * D3Q19 4 (FP32) or 8 (16-bit: a kernel that stages 256-node row segments in shared
 * memory, bit-identical to 4-node packs). It also sets the width (1, 2 or 4) of the
 * adjoint kernel. */
LBMRV_API int lbmrv_set_kernel_width(lbmrv_t h, int nodes_per_thread);

/* Prescribed relative velocity u~(x, t) = amplitude * u~0(x) * cos(2 pi t / period),
 * evaluated at the time index t of each relaxation; period <= 0 means no time factor.
 *   ut0_dev  device FP32 [d][n] (one plane per component), kept by reference; or, for
 *            D2Q9 only, NULL for the analytic field u~0 = (cos 2pi y/ny, sin 2pi x/nx).
 * Only used with LBMRV_UT_PRESCRIBED. */
LBMRV_API int lbmrv_set_utilde(lbmrv_t h, const float* ut0_dev, double amplitude, double period);

/* Set the state to the equilibrium f_eq(rho, u) at every node and the time to 0:
 * f_eq,j = w_j rho (1 + 3 v_j.u/l^2 + 9/2 (v_j.u)^2/l^4 - 3/2 |u|^2/l^2), the
 * second-order polynomial equilibrium (the paper allows any equilibrium independent
 * of u~, Section 1.2). f_eq is a fixed point of the relaxation for every u~, so it is
 * also the post-relaxation state at time 0.
 *   rho_dev  device FP32 [n], or NULL for rho = 1 everywhere.
 *   u_dev    device FP32 [d][n] (one plane per component), physical units.
 * With the automatic reference (the default, lbmrv_set_reference_auto) the call first
 * reduces the fields to their mean flow on the device and reads it back, so it
 * synchronises the handle's stream; with a fixed reference it is asynchronous.
 * Errors: LBMRV_E_INVAL; LBMRV_E_NONFINITE when the automatic reference meets non-finite
 * fields (the state is then left unchanged); LBMRV_E_CUDA. */
LBMRV_API int lbmrv_init_equilibrium(lbmrv_t h, const float* rho_dev, const float* u_dev);

/* Same from host buffers: copies them into the non-current state buffer on the
 * handle's stream (no allocation), then builds the equilibrium. Pinned host memory is
 * faster. With a fixed reference the call returns once the work is enqueued, and the host
 * buffers may be reused only after the stream has synchronised; with the automatic
 * reference it synchronises once the fields are on the device. */
LBMRV_API int lbmrv_init_equilibrium_host(lbmrv_t h, const float* rho_host, const float* u_host);

/* Advance n >= 0 time steps. Each step is one fused kernel: pull transport of the
 * previous post-relaxation state (relation (transport)), then the relaxation in the
 * frame moving at u~ (relation (relaxationu)) done as
 *   m0 = M(0) f, d = m0 - m_eq(0), f* = f - M(0)^{-1} T(-u~) S T(u~) d
 * with T from Appendix A. Step k relaxes at time index t = k. */
LBMRV_API int lbmrv_step(lbmrv_t h, int64_t n);

/* Density and velocity u = q/rho (relation (rhoq)) of the current state.
 *   rho_dev  device FP32 [n] or NULL;  u_dev  device FP32 [d][n] or NULL. */
LBMRV_API int lbmrv_moments(lbmrv_t h, float* rho_dev, float* u_dev);

/* Same into host buffers; synchronous. Uses the non-current state buffer as staging. */
LBMRV_API int lbmrv_moments_host(lbmrv_t h, float* rho_host, float* u_host);

/* Global sums of the current state, accumulated in FP64: out_host[0] = sum rho,
 * out_host[1..2] = sum q_x, sum q_y (physical units), out_host[3] = number of nodes holding
 * a non-finite value. Node moments are FP32; each thread adds runs of up to 32 of them in
 * FP32 and the runs in FP64, in a fixed order (deterministic). Synchronous. Returns
 * LBMRV_E_NONFINITE (after filling out_host) when out_host[3] > 0. */
LBMRV_API int lbmrv_conserved(lbmrv_t h, double out_host[4]);

/* Same for any lattice with all momentum components: out_host = {sum rho, sum q_x,
 * sum q_y, sum q_z (0 for D2Q9), non-finite nodes}. */
LBMRV_API int lbmrv_conserved3(lbmrv_t h, double out_host[5]);

/* n >= 1 steps (as lbmrv_step), then the sums of lbmrv_conserved3 of the resulting state,
 * taken inside the last step's kernel from the values it stores (rounded to the storage
 * type), so the state is not read a second time (relation (rhoq) summed over the
 * lattice). Fused for D2Q9 at vector kernel widths (nodes per thread >= 2) and for D3Q19
 * at its default widths (FP32: 4 nodes per thread; FP16/BF16: 8); other widths run the
 * step, then lbmrv_conserved3's own pass. The sums are added in a fixed
 * order (deterministic for a given width and GPU), in FP32 runs of 32 node moments added in
 * FP64; they agree with lbmrv_conserved3 of the same state to the rounding of those runs
 * (about 1e-7 relative to a run's magnitude). The first call, and a call after the lattice
 * or width changed, allocates 32-64 bytes per step-kernel block of scratch, kept until
 * lbmrv_destroy. Synchronous. Returns LBMRV_E_NONFINITE (after filling
 * out_host) when non-finite nodes were found, LBMRV_E_INVAL for n < 1. */
LBMRV_API int lbmrv_step_conserved(lbmrv_t h, int64_t n, double out_host[5]);

/* Copy the current stored state (layout above) to / from a device buffer of
 * lbmrv_state_bytes(). set_state also sets the time index to t. */
LBMRV_API int lbmrv_get_state(lbmrv_t h, void* dst_dev);
LBMRV_API int lbmrv_set_state(lbmrv_t h, const void* src_dev, int64_t t);

/* Device pointer of the current state buffer (no copy; valid until the next step). */
LBMRV_API int lbmrv_state_ptr(lbmrv_t h, void** ptr_out);

/* Time index of the current state (number of steps since the last init/set_state). */
LBMRV_API int64_t lbmrv_time(lbmrv_t h);

/* Replace the q relaxation rates (same rules and warning as lbmrv_create); applies to
 * later steps. */
LBMRV_API int lbmrv_set_rates(lbmrv_t h, const double* s);

/* ---------------------------------------------------------------- discrete adjoint
 * Not in the paper: the reverse-mode derivative of the step as this library computes it.
 * With S_k = C_k(P S_{k-1}) (P the pull transport, C_k the relaxation at time k), a loss
 * L(S_N) has the adjoint recursion
 *   mu_k = J_{C_k}(P S_{k-1})^T a_k,  a_N = dL/dS_N,  a_k = P^T mu_{k+1},  dL/dS_0 = P^T mu_1,
 * where P^T is a push (the transpose of the pull). J_C^T is the hand-derived transpose of
 * the shifted relaxation (moments, equilibrium moments, T(u~), S, T(-u~), M(0)^{-1}),
 * including the dependence of u~ = q/rho on the populations. Parameter gradients are
 * summed over nodes and steps in FP64. D2Q9 only (else LBMRV_E_UNSUPPORTED), with any
 * storage type: with FP16 / BF16 storage the checkpoints and recomputed states are the
 * handle's 16-bit states, the adjoint vectors stay FP32, and J_C is the derivative of the
 * FP32 relaxation at the stored states (the rounding to the storage type is taken as the
 * identity). Not for slabs.
 * Memory: sqrt(N)-style checkpointing. lbmrv_forward_checkpointed stores every seg-th
 * state; lbmrv_adjoint recomputes each segment from its checkpoint (one extra forward in
 * total) and walks it backwards. */

/* Bytes of the caller-owned workspace for n steps with checkpoints every seg steps
 * (1 <= seg <= n): ceil(n/seg) + seg - 1 states in the storage type (9 values per node),
 * two FP32 adjoint states (36 bytes per node each), plus accumulators. -1 on invalid
 * arguments. */
LBMRV_API int64_t lbmrv_adjoint_workspace_bytes(lbmrv_t h, int64_t n, int64_t seg);

/* Advance n steps from the current state (time t0) like lbmrv_step, storing the states
 * at t0, t0 + seg, t0 + 2 seg, ... in ws_dev (device, 256-byte aligned, at least
 * lbmrv_adjoint_workspace_bytes). The handle remembers (n, seg, ws, t0) for lbmrv_adjoint.
 * Errors: LBMRV_E_INVAL, LBMRV_E_NOMEM (workspace too small), LBMRV_E_UNSUPPORTED. */
LBMRV_API int lbmrv_forward_checkpointed(lbmrv_t h, int64_t n, int64_t seg, void* ws_dev,
                                         size_t ws_bytes);

/* Reverse sweep of the last lbmrv_forward_checkpointed(n, seg, ws_dev) (same arguments).
 *   dL_dS_dev     device FP32 [9][nx*ny], 16-byte aligned: dL/dS_N, gradient of the loss
 *                 with respect to the stored state after the n steps (e.g. from
 *                 lbmrv_kinetic_energy or lbmrv_moments_vjp). Not modified.
 *   dL_dS0_dev    device FP32 [9][nx*ny] out, 16-byte aligned: dL/dS_0 (may alias nothing
 *                 else).
 *   dL_ds_host    9 doubles out, or NULL: dL/ds_k (0 for the conserved k < 3).
 *   dL_damp_host  1 double out, or NULL: dL/dA for the prescribed mode (0 otherwise).
 *   dL_dut0_dev   device FP32 [2][nx*ny] out, or NULL: dL/du~0(x) for the prescribed mode
 *                 with a caller field or the analytic one (overwritten).
 * Synchronous (returns host values). The handle's current state is not changed.
 * LBMRV_E_INVAL for NULL or unaligned gradient buffers, before any work is queued. */
LBMRV_API int lbmrv_adjoint(lbmrv_t h, int64_t n, int64_t seg, void* ws_dev, size_t ws_bytes,
                            const float* dL_dS_dev, float* dL_dS0_dev, double* dL_ds_host,
                            double* dL_damp_host, float* dL_dut0_dev);

/* The reverse sweep one step at a time, for callers that drive the forward steps themselves
 * (a slab, whose steps need halo exchanges between them). With the forward S_t =
 * C_t(P S_{t-1}) and a loss L(S_N): mu_N = J_{C_N}^T dL/dS_N, mu_t = J_{C_t}^T P^T mu_{t+1},
 * dL/dS_0 = P^T mu_1 (lbmrv_adjoint_gather). */

/* Doubles of the FP64 parameter-gradient accumulators lbmrv_adjoint_step adds to (-1 for a
 * lattice without adjoint). The caller owns them and zeroes them before the first step. */
LBMRV_API int64_t lbmrv_adjoint_acc_doubles(lbmrv_t h);

/* One reverse step at time index t >= 1:
 *   s_prev_dev  S_{t-1} in the handle's storage type and layout (for a slab: with the halo
 *               layers the forward exchange gave it before step t), 16-byte aligned
 *   a_dev       gather = 0: dL/dS_t (FP32 [9][n]); gather = 1: mu_{t+1}, whose transpose-pull
 *               P^T the kernel forms (for a slab: its halo layers filled by
 *               lbmrv_halo_unpack_adjoint)
 *   mu_dev      out: mu_t, FP32 [9][n] (for a slab only the own layers are written)
 *   acc_dev     lbmrv_adjoint_acc_doubles doubles, added to (dL/ds and dL/dA, per block)
 *   dL_dut0_dev optional FP32 [2][n]: dL/du~0 added to (prescribed mode)
 * a, mu and s_prev 16-byte aligned, a != mu. A slab reverses its own layers only.
 * Asynchronous. */
LBMRV_API int lbmrv_adjoint_step(lbmrv_t h, const void* s_prev_dev, int64_t t,
                                 const float* a_dev, int gather, float* mu_dev,
                                 double* acc_dev, float* dL_dut0_dev);

/* Sums of the accumulators: dL_ds_host[9] (0 for the conserved k < 3) and dL_damp_host
 * (either may be NULL). Synchronous. */
LBMRV_API int lbmrv_adjoint_acc_sum(lbmrv_t h, const double* acc_dev, double* dL_ds_host,
                                    double* dL_damp_host);

/* dL/dS_0 = P^T mu_1 into out_dev (FP32 [9][n]; 16-byte aligned, distinct buffers). For a
 * slab, mu_1's halo layers must have been filled by lbmrv_halo_unpack_adjoint. Asynchronous. */
LBMRV_API int lbmrv_adjoint_gather(lbmrv_t h, const float* mu_dev, float* out_dev);

/* Kinetic energy L = 1/2 sum_x |q|^2 / rho of the current state (FP64 sum, synchronous)
 * and, when dL_dS_dev (device FP32 [9][nx*ny]) is not NULL, its gradient dL/dS (with
 * respect to the stored values, in FP32 whatever the storage type). For a slab, over its
 * own layers (the gradient is 0 on the halo layers). */
LBMRV_API int lbmrv_kinetic_energy(lbmrv_t h, double* ke_host, float* dL_dS_dev);

/* Adjoint of lbmrv_moments at the current state: dL/dS from dL/drho (device FP32 [nx*ny]
 * or NULL) and dL/du (device FP32 [2][nx*ny] or NULL). Asynchronous. */
LBMRV_API int lbmrv_moments_vjp(lbmrv_t h, const float* dL_drho_dev, const float* dL_du_dev,
                                float* dL_dS_dev);

/* Adjoint of lbmrv_init_equilibrium(rho, u): from dL/dS_0 (device FP32 [9][nx*ny]) to
 * dL/drho (device FP32 [nx*ny] or NULL) and dL/du (device FP32 [2][nx*ny] or NULL).
 * rho_dev may be NULL (rho = 1), as in lbmrv_init_equilibrium. Asynchronous. */
LBMRV_API int lbmrv_equilibrium_vjp(lbmrv_t h, const float* rho_dev, const float* u_dev,
                                    const float* dL_dS0_dev, float* dL_drho_dev,
                                    float* dL_du_dev);

/* ---------------------------------------------------------------- slab decomposition
 * What is split across GPUs (or handles) is the exact transport of Section 1.1 (relation
 * (transport)): in pull form a node reads population j from x - v_j dt, so each layer of the
 * lattice (D2Q9: a row, the slab axis is y; D3Q19: a z-plane, the axis is z) needs from each
 * neighbouring layer only the populations whose velocity crosses between them: 3 of 9 for
 * D2Q9 (c_y = +-1), 5 of 19 for D3Q19 (c_z = +-1). A slab handle is an ordinary handle whose
 * lattice has m = own layers + 2 layers: layers 1 .. m-2 are its own, layers 0 and m-1 are
 * halo copies of the neighbours' edge layers. Each step: lbmrv_halo_pack, exchange the
 * buffers with the neighbours (the caller's transport: a device copy, NCCL, ...),
 * lbmrv_halo_unpack, lbmrv_step(h, 1). The step runs over the whole slab unchanged; what it
 * computes in the halo layers is never read, since the next exchange overwrites every halo
 * value a step reads. All slabs of one lattice must store relative to one reference
 * (lbmrv_set_reference, e.g. lbmrv_set_reference_sums of the summed lbmrv_flow_sums).
 * Face buffers hold lbmrv_halo_count values of the storage type; value b is the k-th
 * crossing population (ascending population index), k = b / L, at in-layer node i = b % L
 * (L = nx for D2Q9, nx*ny for D3Q19). */

/* Partition of `extent` layers among `ranks` slabs: slab `rank` owns `*count` consecutive
 * layers from global layer `*first`; the first (extent % ranks) slabs own one layer more.
 * Host only. LBMRV_E_INVAL unless 1 <= ranks <= extent and 0 <= rank < ranks. */
LBMRV_API int lbmrv_slab_plan(int64_t extent, int ranks, int rank, int64_t* first,
                              int64_t* count);

/* Values in one face buffer for a slab lattice of the given dims (halo layers included):
 * 3*nx for D2Q9, 5*nx*ny for D3Q19; -1 when dims hold fewer than 3 layers. Host only. */
LBMRV_API int64_t lbmrv_halo_count(int lattice, const int64_t dims[3]);

/* Index maps of one face (side 0: the lower face, layers 0 and 1; side 1: the upper face,
 * layers m-1 and m-2), as element offsets into the state (plane j at j*n, layout above), in
 * buffer order, lbmrv_halo_count entries each (either pointer may be NULL):
 *   send_idx  values lbmrv_halo_pack puts in the face's buffer: the edge layer's
 *             populations moving across the face (c = -1 through the lower face, c = +1
 *             through the upper face);
 *   recv_idx  halo values lbmrv_halo_unpack fills from the buffer received across the
 *             face (c = +1 into layer 0, c = -1 into layer m-1).
 * The buffer a slab sends through its upper face is the one its upper neighbour receives
 * through its lower face, and vice versa. Host only: these maps are the definition the
 * device pack and unpack follow. LBMRV_E_INVAL for bad dims or side. */
LBMRV_API int lbmrv_halo_map(int lattice, const int64_t dims[3], int side, int64_t* send_idx,
                             int64_t* recv_idx);

/* Declare h a slab: its own layers 1 .. m-2 are the global layers first .. first+m-3 of a
 * periodic lattice of `extent` layers along the slab axis (0 <= first < extent, extent >=
 * m-2). Effects: the analytic prescribed field (D2Q9) is evaluated at the global row;
 * lbmrv_conserved[3] and lbmrv_step_conserved sum the own layers only (the latter by a
 * separate pass); the automatic reference is turned off (a slab needs the shared reference,
 * and lbmrv_init_equilibrium on a slab with the automatic reference is LBMRV_E_INVAL);
 * lbmrv_moments still covers every layer; lbmrv_kinetic_energy and lbmrv_adjoint_step
 * cover the own layers; lbmrv_forward_checkpointed / lbmrv_adjoint (which step without
 * exchanges) return LBMRV_E_UNSUPPORTED. LBMRV_E_INVAL for fewer than 3 layers. */
LBMRV_API int lbmrv_set_slab(lbmrv_t h, int64_t first, int64_t extent);

/* Pack the current state's outgoing face values: send_lo_dev for the neighbour below
 * (side 0), send_hi_dev for the neighbour above (side 1), device buffers of
 * lbmrv_halo_count values of the storage type, either may be NULL. Asynchronous on the
 * handle's stream. LBMRV_E_INVAL when h is not a slab. */
LBMRV_API int lbmrv_halo_pack(lbmrv_t h, void* send_lo_dev, void* send_hi_dev);

/* Write received face values into the current state's halo layers: recv_lo_dev holds what
 * the neighbour below packed for its upper face, recv_hi_dev what the neighbour above packed
 * for its lower face (either may be NULL). Asynchronous. LBMRV_E_INVAL when h is not a
 * slab. */
LBMRV_API int lbmrv_halo_unpack(lbmrv_t h, const void* recv_lo_dev, const void* recv_hi_dev);

/* The adjoint exchange of a slab's adjoint vector mu (FP32, the state layout), for the
 * gathers of the reverse sweep: the other way round from the forward exchange. Through the
 * lower face (side 0) a slab sends layer 1's populations with c = +1 and receives c = -1
 * populations into layer 0; through the upper face (side 1) it sends layer m-2's c = -1
 * populations and receives c = +1 populations into layer m-1. As for the forward exchange,
 * what a slab sends through its upper face its upper neighbour receives through its lower
 * face. Buffers: FP32, lbmrv_halo_count values each, NULL skips a face. The maps are host
 * only; pack and unpack are asynchronous; LBMRV_E_INVAL when h is not a slab. */
LBMRV_API int lbmrv_halo_map_adjoint(int lattice, const int64_t dims[3], int side,
                                     int64_t* send_idx, int64_t* recv_idx);
LBMRV_API int lbmrv_halo_pack_adjoint(lbmrv_t h, const float* mu_dev, float* send_lo_dev,
                                      float* send_hi_dev);
LBMRV_API int lbmrv_halo_unpack_adjoint(lbmrv_t h, float* mu_dev, const float* recv_lo_dev,
                                        const float* recv_hi_dev);

/* FP64 sums {sum rho, sum rho u_x, sum rho u_y, sum rho u_z (0 for D2Q9)} of initial fields
 * (laid out as for lbmrv_init_equilibrium; rho_dev NULL: 1) over the handle's own nodes (a
 * slab's own layers). Summed over the slabs, they give the shared mean-flow reference.
 * Synchronous. */
LBMRV_API int lbmrv_flow_sums(lbmrv_t h, const float* rho_dev, const float* u_dev,
                              double out_host[4]);

/* lbmrv_set_reference(h, rho_ref, U) with U = sums[1..d] / sums[0] (sums as from
 * lbmrv_flow_sums). LBMRV_E_INVAL when sums[0] <= 0, LBMRV_E_NONFINITE for non-finite
 * sums. */
LBMRV_API int lbmrv_set_reference_sums(lbmrv_t h, double rho_ref, const double sums[4]);

/* The same sums as lbmrv_conserved for a caller-owned D2Q9 state, with no handle and no
 * device allocation. The paper has no counterpart: this exists for callers that cannot
 * allocate when they need the check (an allocator that owns all device memory, a loop
 * where cudaMalloc would synchronise the device, a monitor of a buffer it did not
 * create). Scratch comes from a fixed 38,912-byte array in the library's device image,
 * present on every GPU that loads the library until the process exits.
 *   state_dev  device state in the layout above (9 planes of nx*ny, storage type).
 *   storage    LBMRV_FP32 / LBMRV_FP16 / LBMRV_BF16; rho_ref the stored offset (the
 *              state is read with a zero reference velocity; for a state stored with
 *              lbmrv_set_reference(rho_ref, U), add nx*ny*rho_ref*U to the momentum sums).
 *   dims       {nx, ny, 1} (any other depth: LBMRV_E_INVAL); nx*ny must be below 2^31
 *              (larger sizes: LBMRV_E_INVAL).
 *   out_dev    4 device doubles: sum rho, sum q_x, sum q_y, non-finite node count.
 *   stream     cudaStream_t to enqueue on (NULL: the legacy default stream).
 * Asynchronous; allocates nothing (no cudaMalloc, no cudaFree). The first call on a
 * device looks up the scratch array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture. The address is kept per device and looked
 * up again when the device's context has changed (after cudaDeviceReset, for example);
 * make the first call after such a reset before any stream capture too. Every call
 * shares the one scratch array:
 * calls that overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller. Each call overwrites all the scratch it reads, so nothing
 * needs clearing. Returns LBMRV_OK, LBMRV_E_INVAL or LBMRV_E_CUDA (no message is kept,
 * as there is no handle). */
LBMRV_API int lbmrv_conserved_noalloc(const void* state_dev, int storage, const int64_t dims[3],
                                      double lambda, double rho_ref, double* out_dev,
                                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBMRV_H */
