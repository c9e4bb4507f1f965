/*
 * adi_maxwell.h -- C-ABI of the GB300 (sm_103a) ADI isogeometric Maxwell stepper.
 *
 * The method is the alternating-direction-implicit (ADI) time scheme with
 * B-spline (IGA) discretisation of Paszynski, Los and Munoz-Matute,
 * "Alternating directions implicit higher-order finite element method for
 * simulations of time-dependent electromagnetic wave propagation in
 * non-regular biological tissues" (arXiv 2103.06998):
 *
 *   dE/dt = eps^-1 curl H,  dH/dt = -mu^-1 curl E  on (0,1)^3 with
 *   E x n = 0 and H . n = 0 on the boundary        (section "Alternating
 *   directions splitting for Maxwell equations", first system of equations),
 *
 * split as curl = C1 - C2 and advanced in two half steps (eqs. scheme1a-1d),
 * discretised as eqs. discrete1-discrete4 with 1D mass, stiffness and
 * advection matrices on a regular patch of n_x x n_y x n_z elements of degree
 * p, and solved by three banded 1D systems per E component (section
 * "Incorporating non-regular material data", Appendix eqs. split1/split2).
 * Material data are attached to the test functions (rows).
 *
 * Conventions shared by all calls:
 *  - Coefficient arrays are [component][z][y][x], x fastest, N_d = n_d + p
 *    coefficients per axis, N_c = N_x N_y N_z per component.  The six
 *    components are ordered E1, E2, E3, H1, H2, H3.
 *  - Per-element material arrays are [z][y][x] with n_x n_y n_z entries.
 *  - The caller owns every host pointer; the library copies what it needs and
 *    keeps no caller pointer after a call returns, except the host buffers of
 *    the asynchronous transfers (adi_set_fields_async, adi_fields_async), which
 *    stay in use until adi_sync returns.
 *  - A handle owns all device memory it allocates; adi_destroy frees it.
 *  - No call aborts or throws.  Failures return a status other than ADI_OK and
 *    set a message readable with adi_last_error(h) (adi_last_error(NULL) for
 *    calls without a handle, a NULL handle, or a failed create).
 *  - Errors common to the calls that take a handle: ADI_EINVAL for a NULL
 *    handle or an argument outside its documented range (the message names
 *    it), ADI_ECUDA when a CUDA call fails (ADI_ENOMEM when it is an
 *    allocation).  Each call lists the others it can return.
 *  - Work is issued on the handle's CUDA stream (adi_set_stream; default: the
 *    library's own non-blocking stream).  Calls that return host data
 *    synchronise that stream.
 *  - A handle is used by one host thread at a time.
 */
#ifndef ADI_MAXWELL_H
#define ADI_MAXWELL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adi_ctx* adi_handle;

typedef enum {
  ADI_OK = 0,
  ADI_EINVAL = 1,   /* invalid argument (sizes, p, dt, material <= 0, null pointer) */
  ADI_ENOMEM = 2,   /* device or host allocation failed */
  ADI_ECUDA = 3,    /* a CUDA call failed (message has the CUDA error string) */
  ADI_ESTATE = 4,   /* call out of order (e.g. adi_step before adi_factor) */
  ADI_ENUMERIC = 5, /* NaN or Inf found in an input or an output */
  ADI_ETIMEOUT = 6  /* a bounded device wait gave up */
} adi_status;

/* Arithmetic of the time step.
 *  ADI_PREC_FP32, ADI_PREC_FP64: every kernel in that type.
 *  ADI_PREC_MIXED: FP32 state and line solves; in each E half step the
 *  right-hand side is contracted from field tiles rounded to BF16 with FP32
 *  accumulation, giving E*; then one refinement: the residual
 *  r = RHS - T E* of the E system T E = RHS is evaluated to about 48
 *  significant bits (from the FP32 state), T delta = r is solved in FP32 and
 *  E = E* + delta.  The residual's arithmetic is compensated double-float on
 *  the FP32 pipe (TwoSum, TwoProduct by FMA) by default, or FP64 with
 *  mixed_fp64_residual = 1.  The 1D factorisations are FP64 in every mode.
 *  The paper states no precision; this mode is an addition. */
enum { ADI_PREC_FP64 = 0, ADI_PREC_FP32 = 1, ADI_PREC_MIXED = 2 };

/* Where the per-element material enters the right-hand sides (section
 * "Incorporating non-regular material data").  ADI_RHS_ROW (default, the
 * paper's reading): every row rst is scaled by its coefficients a, b, c, d
 * formed from the hat values eps^, mu^, sigma^ of test function rst.
 * ADI_RHS_QUAD: each right-hand-side integral carries the element's own
 * coefficients inside the integrand, sum_e kappa_e int_e (...) B_rst with
 * kappa_e = a_e, b_e, c_e, d_e formed from the element's eps, mu, sigma by the
 * same formulas (the dipole row uses b of the element that holds it).  The
 * left-hand sides stay row-scaled in both readings (that keeps their Kronecker
 * structure, hence the line solves); the two readings agree for uniform
 * material.  With uniform mu the H half steps are the same in both. */
enum { ADI_RHS_ROW = 0, ADI_RHS_QUAD = 1 };

typedef struct {
  int precision;        /* ADI_PREC_FP32 (default), ADI_PREC_FP64 or ADI_PREC_MIXED */
  int use_graph;        /* 1 (default): adi_step replays a captured CUDA graph of one step */
  int mixed_no_refine;  /* ADI_PREC_MIXED only: 1 skips the refinement (E = E*, for error studies) */
  int mixed_fp64_residual; /* ADI_PREC_MIXED only: 1 evaluates the residual in FP64 (default 0: float-float) */
  int rhs_material;     /* ADI_RHS_ROW (default) or ADI_RHS_QUAD (not with ADI_PREC_MIXED; p <= 3 in FP64) */
  int serial_chains;    /* 0 (default): the line solves of the three E components of a half step run as three
                           concurrent chains on streams of the handle (parallel branches of the step's graph);
                           1: one after another on the handle's stream.  Same results bit for bit. */
  int reserved[2];      /* must be 0 */
} adi_options;

/* Create a problem on the unit cube.
 *  nx, ny, nz >= 1 elements per axis; 1 <= p <= 4 (B-spline degree, C^{p-1});
 *  dt > 0 is the full time step tau (each half step advances tau/2);
 *  eps, mu, sigma: per-element relative permittivity, permeability and
 *  conductivity ([z][y][x], n_x n_y n_z doubles each); NULL means 1, 1, 0.
 *  eps and mu must be > 0 (first system of equations: eps, mu >= delta > 0)
 *  and sigma >= 0, else ADI_EINVAL.  opt may be NULL (defaults).
 *  Per-element values become per-test-function values by the support-weighted
 *  mean  v_rst = sum_e v_e W_e / sum_e W_e,  W_e = prod_d int_{e_d} B_{r_d}
 *  (the paper attaches material to test functions but does not say how voxel
 *  data map to them; this is the reading used).  Conductivity enters as
 *  eps dE/dt + sigma E = curl H - J, trapezoidal over each half step.
 *  On success *out is a new handle with all fields zero at t = 0. */
adi_status adi_create(int nx, int ny, int nz, int p, double dt,
                      const double* eps, const double* mu, const double* sigma,
                      const adi_options* opt, adi_handle* out);

/* adi_create on non-uniform elements (section "Variational formulation": the
 * 1D matrices are defined for any open knot vector; bandwidth stays 2p + 1).
 *  breaks_x, breaks_y, breaks_z (host, caller-owned, copied): the element
 *  boundaries of each axis, n_d + 1 doubles, 0 = x_0 < x_1 < ... < x_{n_d} = 1
 *  (NULL: uniform elements on that axis); the knot vector repeats the end
 *  points p + 1 times.  Material, source position and plane coordinates refer
 *  to these elements (a point on an element boundary belongs to the element on
 *  its right).  Kernels use the constant interior stencil only on rows whose
 *  band rows agree with it (a uniform core), the band tables elsewhere.
 * Errors as adi_create; ADI_EINVAL also for boundaries that are not strictly
 * increasing from 0 to 1.  The batched instances, the corrector and
 * adi_cfl_dt_noalloc use uniform elements. */
adi_status adi_create_knots(int nx, int ny, int nz, int p, double dt, const double* breaks_x,
                            const double* breaks_y, const double* breaks_z, const double* eps, const double* mu,
                            const double* sigma, const adi_options* opt, adi_handle* out);

/* Host only (no device, no handle): the 1D matrices of one axis exactly as
 * adi_create / adi_create_knots build them (definitions after eq. discrete4:
 * M[l][i] = int B_i B_l, S[l][i] = int B_i' B_l', A[l][i] = int B_i' B_l,
 * B[l][i] = int B_i B_l', row l the test function; Gauss-Legendre with p + 1
 * points per element, exact for these integrands, in FP64), in band form: row
 * k of X at out[k (2p+1) + d] = X[k][k + d - p], k = 0 .. N-1, N = n + p
 * (entries outside the matrix are 0).
 *  n >= 1, 1 <= p <= 4; breaks: n + 1 element boundaries as in
 *  adi_create_knots, or NULL (uniform elements).
 *  M, S, A, B (host, caller-owned; any may be NULL to skip it): N (2p+1)
 *  doubles each.  inner (host, caller-owned, may be NULL): 2 ints, the first
 *  and last row whose band rows the kernels replace by the constant interior
 *  stencil (inner[0] > inner[1]: none).
 * Errors: ADI_EINVAL (n, p or breaks), ADI_ENOMEM (host allocation). */
adi_status adi_axis_bands(int n, int p, const double* breaks, double* M, double* S, double* A, double* B,
                          int* inner);

/* Host only: two further per-axis tables the solver derives from the 1D basis.
 *  G (host, caller-owned, may be NULL): N (p+1) doubles, G[r (p+1) + a] = the
 *  integral of B_r over element r - p + a (0 where that element does not
 *  exist); these weights turn per-element material into per-test-function
 *  values (see adi_create).
 *  lam (host, may be NULL): the largest eigenvalue of M_D^{-1} S_D, M and S
 *  with the first and last basis functions removed; adi_cfl_dt sums it over
 *  the three axes (the explicit-scheme limit, a reference scale for choosing
 *  the time step).
 *  n, p, breaks as adi_axis_bands.  Errors: ADI_EINVAL, ADI_ENOMEM. */
adi_status adi_axis_tables(int n, int p, const double* breaks, double* G, double* lam);

/* Host only: the per-element blocks of the 1D matrices of one axis, which the
 * right-hand side with per-element material inside the integrals
 * (ADI_RHS_QUAD) contracts element by element:
 *  loc[((e 4 + op) (p+1) + a) (p+1) + b] = the integral over element e of the
 *  op's integrand (op 0..3: M, S, A, B as in adi_axis_bands) for test function
 *  e + a and trial function e + b; the bands are the sums of these blocks.
 *  n, p, breaks as adi_axis_bands; loc (host, caller-owned): 4 n (p+1)^2
 *  doubles.  Errors: ADI_EINVAL, ADI_ENOMEM. */
adi_status adi_axis_element_matrices(int n, int p, const double* breaks, double* loc);

/* Host only: the LU factors of the 1D mass matrix M of one axis exactly as
 * adi_factor computes them (no pivoting; M is symmetric positive definite),
 * for the full matrix (reduced = 0: rows and columns 0 .. N-1) or the
 * Dirichlet-reduced one (reduced = 1: 1 .. N-2, the first and last basis
 * functions removed).  Over those rows, M = L D U with L unit lower and U unit
 * upper triangular of bandwidth p and D diagonal:
 *  L[k p + q - 1] = L[k][k - q], U[k p + q - 1] = U[k][k + q] (q = 1..p),
 *  inv_d[k] = 1 / D[k]; rows outside the range are 0.
 *  n, p, breaks as adi_axis_bands; L, U (host, caller-owned): N p doubles,
 *  inv_d: N doubles.  Errors: ADI_EINVAL, ADI_ENOMEM. */
adi_status adi_axis_mass_lu(int n, int p, const double* breaks, int reduced, double* L, double* inv_d, double* U);

/* Host only: the p + 1 B-splines of one axis that are nonzero at x0 in [0, 1]
 * and their values there, as the point source uses them (the dipole's spatial
 * factor, section "Incorporating non-regular material data"): *first = e, the
 * element holding x0 (a point on an element boundary belongs to the element on
 * its right, x0 = 1 to the last), vals[a] = B_{e+a}(x0), a = 0..p.
 *  n, p, breaks as adi_axis_bands; vals (host, caller-owned): p + 1 doubles.
 * Errors: ADI_EINVAL (also x0 outside [0, 1]), ADI_ENOMEM. */
adi_status adi_axis_point_basis(int n, int p, const double* breaks, double x0, int* first, double* vals);

/* Factor the mass matrices of every axis (full and Dirichlet-reduced, without
 * pivoting, in FP64) from the 1D matrices M, S, A (B = A^T) that adi_create
 * built by Gauss-Legendre quadrature in FP64 (definitions after eq.
 * discrete4), and upload the bands and factors in the working precision.
 * Must precede adi_step (else ADI_ESTATE).  Errors: ADI_ECUDA, ADI_ENOMEM. */
adi_status adi_factor(adi_handle h);

/* Change the time step; the row coefficients are rebuilt and adi_factor must
 * be called again before the next adi_step (else ADI_ESTATE).
 * Errors: ADI_EINVAL (dt not finite and > 0). */
adi_status adi_set_dt(adi_handle h, double dt);

/* Use the given cudaStream_t (NULL = legacy default stream; not owned) for all
 * later work.  Synchronises the current stream and the asynchronous-transfer
 * streams first.  On the legacy default stream adi_step cannot capture a CUDA
 * graph and issues the kernels one by one. */
adi_status adi_set_stream(adi_handle h, void* cuda_stream);

/* Copy 6 N_c doubles (host) into the state and set the time to t.  The
 * coefficients that the boundary conditions fix to zero (E_i in the two
 * directions other than i, H_i in direction i: first and last B-spline) are
 * set to zero.  NaN/Inf in EH gives ADI_ENUMERIC and leaves the state and the
 * time unchanged (the check runs on the device; the call synchronises the
 * handle's stream to read it).  A page-locked EH (pinned or registered) is read
 * by the device directly; other memory is copied to a staging buffer first.  A
 * partial step (adi_substep) in progress is discarded. */
adi_status adi_set_fields(adi_handle h, const double* EH, double t);

/* Point dipole J = amp g(t) delta(x - x0) e_comp (comp 0, 1, 2 = E1, E2, E3),
 * g(t) = sin(2 pi f0 (t - t0)) exp(-((t - t0)/s)^2).  Enters the E rows as
 * -b (J, B_rst) at the mid time of each half step.  Not part of the paper's
 * equations.  amp = 0 removes the source.  Errors: ADI_EINVAL (x0 outside
 * [0,1]^3, comp not 0..2, amp, f0 or t0 not finite, s not > 0). */
adi_status adi_set_source(adi_handle h, double x0, double y0, double z0, int comp,
                          double amp, double f0, double t0, double s);

/* Advance n >= 1 full time steps (eqs. scheme1a-1d: E half step 1, H half step
 * 1, E half step 2, H half step 2).  Asynchronous on the handle's stream.
 * Errors: ADI_EINVAL (n < 1), ADI_ESTATE (before adi_factor). */
adi_status adi_step(adi_handle h, int n);

/* Run one sub-solve only: which = 0 (E, half step 1), 1 (H, half step 1),
 * 2 (E, half step 2), 3 (H, half step 2, also advances the time by tau).
 * Four calls in order equal one adi_step.  For testing.  Errors: ADI_EINVAL
 * (which outside 0..3), ADI_ESTATE (before adi_factor). */
adi_status adi_substep(adi_handle h, int which);

/* Copy the state to 6 N_c host doubles (working precision widened) and the
 * current time to *t (t may be NULL).  Synchronises the stream.  Returns
 * ADI_ENUMERIC if any value is NaN/Inf (the data are still copied).  A
 * page-locked EH is written by the device directly. */
adi_status adi_fields(adi_handle h, double* EH, double* t);

/* adi_set_fields and adi_fields with 6 N_c floats on the host side (the same
 * layout, checks and synchronisation).  In all four calls EH must be aligned
 * to its element size (else ADI_EINVAL, nothing is read or written).  For a handle whose state is FP32
 * (ADI_PREC_FP32, ADI_PREC_MIXED) they move exactly the state's values in half
 * the bytes of the double forms; for an FP64 handle the values are rounded to
 * float on the way out and widened on the way in. */
adi_status adi_set_fields_f32(adi_handle h, const float* EH, double t);
adi_status adi_fields_f32(adi_handle h, float* EH, double* t);

/* Asynchronous host transfers, for loops that keep the host link busy while
 * the GPU steps (for example a service that sets a state, steps it and reads it
 * back, over and over).  EH must be page-locked host memory (pinned or
 * registered) aligned to elem_bytes (4: floats, 8: doubles; the layout of
 * adi_set_fields); else ADI_EINVAL.  Neither call waits: the caller leaves EH
 * unchanged (set) or unread (read) until adi_sync returns.  The first call
 * allocates two device arrays of 6 N_c elem_bytes bytes (a later call with
 * larger elements replaces them); ADI_ENOMEM if that fails.
 *   adi_set_fields_async copies EH to device memory on an input stream of the
 *   handle as soon as the previous asynchronous set has been applied (so while
 *   the steps enqueued before it run), then applies it to the state, with the
 *   time t, after everything enqueued on the handle before the call.  A NaN or
 *   Inf in EH leaves the state and its device clock unchanged (the handle's
 *   host-side time follows the call regardless) and makes the next adi_sync
 *   return ADI_ENUMERIC.
 *   adi_fields_async takes the state after everything enqueued before it into
 *   device memory and copies it to EH on an output stream while the work
 *   enqueued after the call runs; a NaN or Inf makes the next adi_sync return
 *   ADI_ENUMERIC (the data are still written).
 * Everything enqueued on the handle after either call is ordered after it.  In
 * the sequence set, step, read, set, step, read, ... the copy of each set runs
 * during the step before it and the copy of each read during the step after
 * it, on the two directions of the host link.
 * No counterpart in the paper. */
adi_status adi_set_fields_async(adi_handle h, const void* EH, int elem_bytes, double t);
adi_status adi_fields_async(adi_handle h, void* EH, int elem_bytes);

/* Copy the state, in the working precision (float or double as created), to
 * 6 N_c elements of device memory at dev_ptr (caller-owned, the dense layout
 * of adi_set_fields), on cuda_stream (NULL = the handle's stream; another
 * stream first waits, on the host, for the handle's stream).  Asynchronous.
 * Errors: ADI_EINVAL (dev_ptr NULL). */
adi_status adi_fields_device(adi_handle h, void* dev_ptr, void* cuda_stream);

/* Norms of the current state as functions on the unit cube: the paper plots the
 * L2 and H1 norms of E and H over time for the head simulation (section
 * "Incorporating non-regular material data", Figure head_norms) and measures the
 * manufactured-solution errors in the L2 and H(curl) norms (section "Numerical
 * code verification with manufactured solution").
 *  out[6] (host) = { ||E||_L2, ||H||_L2, ||E||_H1, ||H||_H1, ||E||_Hcurl, ||H||_Hcurl },
 *  ||u||_H1^2 = ||u||_L2^2 + sum_i ||grad u_i||^2, ||u||_Hcurl^2 = ||u||_L2^2 + ||curl u||^2.
 * Computed on the device as quadratic forms of the 1D matrices (c . (M(x)M(x)M) c
 * and the like; exact integrals of the B-spline fields), summed in FP64 from
 * the working precision; uses the right-hand-side scratch arrays, so it runs
 * in stream order between steps.  Synchronises the handle's stream.
 * Errors: ADI_EINVAL, ADI_ECUDA, ADI_ENUMERIC (NaN or Inf in the state). */
adi_status adi_norms(adi_handle h, double* out);

/* Values of one state component on a uniform grid of a coordinate plane (the
 * paper's field pictures are cross sections along an OYZ plane, Figures head2
 * and head3), written headless to a host buffer.
 *  comp: 0..5 = E1, E2, E3, H1, H2, H3; axis: 0 (plane x = pos), 1 (y), 2 (z);
 *  pos in [0, 1]; the grid points are u_j = j / (nu - 1), v_k = k / (nv - 1) over
 *  the two other axes in x, y, z order (axis 0: u = y, v = z);
 *  out (host, caller-owned): nu * nv doubles, out[k * nu + j].
 * nu, nv >= 2 and (1 + nu + nv)(p + 2) + nu nv <= 6 N_c (the handle's staging
 * buffer holds the point tables and the result).  Synchronises the handle's
 * stream.  Errors: ADI_EINVAL, ADI_ECUDA. */
adi_status adi_plane(adi_handle h, int comp, int axis, double pos, int nu, int nv, double* out);

/* Explicit-scheme stability limit used to choose dt (not in the paper):
 * 2 / (c_max sqrt(lambda_x + lambda_y + lambda_z)), lambda_d the largest
 * eigenvalue of M^-1 S on axis d (Dirichlet-reduced), c_max =
 * 1/sqrt(min_rows eps^ mu^).  Returns a negative value on error. */
double adi_cfl_dt(adi_handle h);

/* Allocation-free variant of adi_cfl_dt for callers that cannot allocate
 * device memory (the paper has no counterpart; this is a library service).
 * Who needs it: services that give all device memory to their own pool at
 * start-up and forbid later cudaMalloc/cudaFree, real-time loops that must not
 * block in the allocator, and plug-ins of a host application that owns every
 * device allocation.  adi_create allocates
 * the whole state, so such callers cannot get the explicit time-step limit
 * from a handle at that point; this call computes the same value as
 * adi_cfl_dt of a handle created from the same nx, ny, nz, p, eps and mu.
 *  d_eps, d_mu: per-element eps and mu in DEVICE memory ([z][y][x], doubles,
 *  owned by the caller, read only).  *dt_out (host) receives the limit.
 *  cuda_stream: the stream to run on (NULL = legacy default stream); the call
 *  synchronises it before returning.
 * No device memory is allocated or freed: the scratch (the 1D element-integral
 * tables and a running minimum) is one file-scope device array of 8192
 * doubles (64 KiB) that every GPU which loads the library keeps until the
 * process exits.  Sizes with (nx + ny + nz + 3p) * (p + 1) > 8184 are rejected
 * with ADI_EINVAL before any GPU work.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the one
 * array and each call re-initialises what it reads, so calls that overlap on
 * the GPU (different streams, or host threads on the same device) race and
 * must be serialised by the caller.  Errors: ADI_EINVAL (NULL pointer, sizes),
 * ADI_ECUDA, ADI_ENUMERIC (some eps or mu element negative, zero, NaN or Inf:
 * every element is checked on the device); message via adi_last_error(NULL). */
adi_status adi_cfl_dt_noalloc(int nx, int ny, int nz, int p, const double* d_eps, const double* d_mu,
                              void* cuda_stream, double* dt_out);

/* Lines per CTA of the line-solve kernels: 8, 16, 32 or 64, or 0 for the
 * default (the largest that leaves room for two CTAs per SM).  A width whose
 * shared memory does not fit falls back to the default.  Used by the
 * autotuner of the batched mode; results do not depend on it.  Errors:
 * ADI_EINVAL (another width). */
adi_status adi_set_line_tile(adi_handle h, int lines);

/* ---------------------------------------------------------------- batches
 * Many independent problems of different sizes, materials, degrees and time
 * steps stepped together (the paper steps one patch; batching is a library
 * service).  Each instance is an ordinary handle owned by the batch: set its
 * fields, source and time step through adi_batch_handle and the calls above.
 * adi_batch_step advances every instance by n steps: one step of all instances
 * is captured once as a CUDA graph whose branches are the instances' sub-step
 * kernels on their own streams (forked from and joined to the batch stream),
 * so the GPU runs small instances concurrently; the graph is replayed n times.
 * Results equal those of each instance stepped alone, bit for bit.  Batch
 * calls report failures in adi_last_error(NULL) (a NULL batch is ADI_EINVAL);
 * a failing instance call passes its status through, with the instance's
 * message. */
typedef struct adi_batch_ctx* adi_batch;
typedef struct {
  int nx, ny, nz, p; /* as adi_create */
  double dt;
  const double* eps; /* per-element material, NULL = 1, 1, 0 */
  const double* mu;
  const double* sigma;
} adi_instance_desc;

/* Create count >= 1 instances (adi_create each, same options).  On failure
 * nothing is kept and the message is in adi_last_error(NULL). */
adi_status adi_batch_create(int count, const adi_instance_desc* desc, const adi_options* opt, adi_batch* out);
/* The handle of instance i (owned by the batch: do not destroy it).
 * Errors: ADI_EINVAL (i outside 0 .. count-1, h NULL). */
adi_status adi_batch_handle(adi_batch b, int i, adi_handle* h);
/* Run the batch on the given cudaStream_t (not owned; NULL = the batch's own stream). */
adi_status adi_batch_set_stream(adi_batch b, void* cuda_stream);
/* adi_factor of every instance. */
adi_status adi_batch_factor(adi_batch b);
/* Advance every instance by n >= 1 steps (asynchronous on the batch stream;
 * the instances' own streams are synchronised first and later calls on an
 * instance are ordered after the batch).  Errors: ADI_EINVAL (n < 1),
 * ADI_ESTATE (an instance not factored), ADI_ECUDA. */
adi_status adi_batch_step(adi_batch b, int n);
/* Block until the batch stream and every instance are idle (adi_sync of each
 * instance): ADI_ETIMEOUT if a bounded device wait gave up, ADI_ENUMERIC as
 * adi_sync, ADI_ECUDA. */
adi_status adi_batch_sync(adi_batch b);
/* Pick the line-tile width of every instance by timed trials (8..64 lines,
 * three steps each, on the instance alone) unless cache_path (may be NULL)
 * already holds a choice for its (p, N_x, N_y, N_z, precision); new choices
 * are appended to cache_path.  The fields are restored afterwards.
 * Errors: ADI_ESTATE (an instance not factored), and those of adi_fields,
 * adi_set_fields and adi_step on an instance. */
adi_status adi_batch_autotune(adi_batch b, const char* cache_path);
/* Release the batch and all its instances.  NULL is ignored. */
void adi_batch_destroy(adi_batch b);

/* Block until all work on the handle's streams is done.  Returns ADI_ETIMEOUT
 * when a bounded device wait of a kernel gave up since the last report (an
 * asynchronous copy was not delivered within its iteration limit; the kernel
 * left its results unwritten and returned instead of hanging); the status is
 * reported once and then cleared.  adi_fields reports it the same way.  Then
 * ADI_ENUMERIC when an asynchronous transfer since the last report met a NaN
 * or Inf (reported once). */
adi_status adi_sync(adi_handle h);

/* Diagnostic (not in the paper): run one of the kernels' bounded waits on a
 * barrier that never completes, asynchronously on the handle's stream, so the
 * time-out path can be tested without a fault.  which: 0 = the E right-hand
 * side's tile wait, 1 = the x line solves' bulk-copy wait; budget: iterations
 * before giving up (0 .. 2^22).  No copy is issued, so nothing is in flight when
 * the wait gives up.  The next adi_sync returns ADI_ETIMEOUT, the one after it
 * ADI_OK; the handle stays usable.  Errors: ADI_EINVAL (which, budget). */
adi_status adi_wait_selftest(adi_handle h, int which, int budget);

/* Per-kernel timing.  With profiling on, every kernel launch of adi_step /
 * adi_substep is bracketed by CUDA events on the handle's stream (graphs are
 * not used while it is on).  adi_kernel_stats fills up to max entries with
 * the kernel family name (static string), launch count, and summed device
 * milliseconds since profiling was switched on, and sets *count; it
 * synchronises the stream. */
typedef struct {
  const char* name;
  long long launches;
  double total_ms;
  double bytes_per_launch; /* algorithmic bytes moved by one launch */
} adi_kernel_stat;
adi_status adi_set_profiling(adi_handle h, int on);
adi_status adi_kernel_stats(adi_handle h, adi_kernel_stat* out, int max, int* count);

/* Sizes: N_x, N_y, N_z, and bytes of one working-precision element (host
 * ints, any may be NULL).  Errors: ADI_EINVAL (NULL handle). */
adi_status adi_dims(adi_handle h, int* Nx, int* Ny, int* Nz, int* elem_bytes);

/* Release everything owned by h.  NULL is ignored. */
void adi_destroy(adi_handle h);

/* Message of the last failure on h (or of the last failed adi_create when h
 * is NULL).  Never NULL. */
const char* adi_last_error(adi_handle h);

/* Static name of a status code. */
const char* adi_status_string(adi_status s);

#ifdef __cplusplus
}
#endif
#endif /* ADI_MAXWELL_H */
