// Internal declarations shared by the C-ABI (adi_capi.cpp), the host setup
// (setup_host.cpp) and the CUDA kernels (adi_kernels.cu).
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the driver entry point is looked up at run time)
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/adi_maxwell.h"

namespace adi {

constexpr int kMaxP = 4;
constexpr int kMaxTerms = 12;
constexpr int kMaxResidTerms = 18;  // E right-hand side (12) and T E* (6) of the mixed-mode residual

// ---------------------------------------------------------------- host setup
struct Axis1D {
  int n = 0, p = 0, N = 0;
  std::vector<double> breaks;      // element boundaries x_0 = 0 < ... < x_n = 1 (empty: uniform)
  std::vector<double> M, S, A, B;  // bands, row k: [k*(2p+1) + d] = X[k][k+d-p]
  std::vector<double> G;           // G[r*(p+1) + a] = int over element r-p+a of B_r
  // rows inner_lo .. inner_hi (inside 2p .. N-1-2p) have the band rows of the middle
  // row (the interior stencil; all of 2p .. N-1-2p for uniform elements)
  int inner_lo = 1, inner_hi = 0;
};
struct LuConst {  // rows lo..hi of a mass LU share the factors v (in the working precision)
  int lo = 1, hi = 0;
  double v[3 * kMaxP + 1] = {};
};
struct BandLU {
  int N = 0, p = 0, lo = 0, hi = 0;
  std::vector<double> L, inv_d, U;  // L[k*p+q-1], U[k*p+q-1] for q = 1..p
};
// breaks: n + 1 element boundaries from 0 to 1, or NULL for uniform elements
void build_axis(int n, int p, Axis1D& ax, const double* breaks = nullptr);
void band_lu(const std::vector<double>& base, const std::vector<double>* stiff, int N, int p,
             int lo, int hi, BandLU& out);
double lambda_max(const Axis1D& ax);
int point_basis(int n, int p, double x0, double* vals);
// the element of ax that holds x0 (a boundary point belongs to the element on its
// right, x0 = 1 to the last) and the p + 1 B-splines nonzero there, at x0
int point_basis(const Axis1D& ax, double x0, double* vals);
// per-element blocks of M, S, A, B: loc[((e*4 + op)*(p+1) + test)*(p+1) + trial]
void element_matrices(const Axis1D& ax, std::vector<double>& loc);

// ---------------------------------------------------------- device structures
// Operator codes of one Kronecker factor.
enum Op : int { OP_M = 0, OP_S = 1, OP_A = 2, OP_B = 3 };
// Row coefficient selecting a, b, c, d or 1.
enum Coef : int { CF_ONE = 0, CF_A = 1, CF_B = 2, CF_C = 3, CF_D = 4 };

template <typename T>
struct AxisDev {
  const T* band[4];     // M, S, A, B bands (N x (2p+1))
  const T* luL[2];      // mass LU, [0] full, [1] Dirichlet-reduced
  const T* luInv[2];
  const T* luU[2];
  int N;
  // rows inner_lo .. inner_hi of M, S, A, B equal the interior stencil inner[op]
  T inner[4][2 * kMaxP + 1];
  int inner_lo, inner_hi;
  // rows lu_lo[f] .. lu_hi[f] of the mass LU f have the factors luc[f] in T:
  // [L(1..p), 1/pivot, U(1..p)]
  T luc[2][3 * kMaxP + 1];
  int lu_lo[2], lu_hi[2];
};

struct Term {
  int field;   // index into RhsParams::fields
  int out;     // output component 0..2
  int op[3];   // Op for x, y, z
  int coef;    // Coef
  float sign;  // +1 or -1
};

// Interior (translation-invariant) stencils of M, A, B on one axis: rows
// 2p .. N-1-2p of the band tables are all equal for open uniform knots.
template <typename T>
struct Stencils {
  T w[3][2 * kMaxP + 1];  // [M, A, B][tap]
  int lo, hi;             // interior rows: lo <= row <= hi (lo > hi: none)
};

template <typename T>
struct RhsParams {
  const T* fields[9];
  const T* coef[5];  // [CF_A], [CF_B], [CF_C], [CF_D] (index 0 unused)
  T* out[3];
  AxisDev<T> ax[3];
  Term terms[kMaxTerms];
  int nterms;
  int nfields;
  int Nx, Ny, Nz;
  int pitch;           // elements between consecutive x rows (>= Nx, multiple of 4)
  // point source (E rows only): comp < 0 disables
  int src_comp;
  int src_i0[3];
  T src_w[3][kMaxP + 1];
  double src_amp, src_f0, src_t0, src_s;
  double tau, t_frac;  // mid time = clock.t0 + (clock.step + t_frac) * tau
  const double* clock_t0;
  long long* clock_step;
  int advance_clock;   // 1: block 0 thread 0 increments the step counter
  Stencils<T> st[3];   // interior stencils per axis (E kernel)
  int* err;            // device status word: bit 0 = a bounded wait gave up
};

// Right-hand side with per-element coefficients inside the integrals: the
// terms of RhsParams, the element blocks of the 1D matrices, the material.
template <typename T>
struct QuadParams {
  const T* fields[9];
  T* out[3];
  const T* loc[3];  // per axis: [e][op M, S, A, B][test][trial]
  const double* eps;
  const double* mu;
  const double* sigma;
  double tau;
  Term terms[kMaxTerms];
  int nterms;
  int n[3];
  int Nx, Ny, Nz, pitch;
  int src_comp;  // < 0: none
  int src_e[3];  // element holding the dipole (its first B-spline per axis)
  T src_w[3][kMaxP + 1];
  double src_amp, src_f0, src_t0, src_s;
  double t_frac;
  const double* clock_t0;
  const long long* clock_step;
};

// TMA descriptors of the six input fields of one E right-hand side launch.
struct TmaMaps {
  CUtensorMap m[6];
};

struct LineParams {
  int dir;        // 0 x, 1 y, 2 z
  int N;          // line length
  long long nlines;
  int Nx, Ny, Nz;
  int pitch;      // elements between consecutive x rows
  int* err;       // device status word: bit 0 = a bounded wait gave up
};

enum LineMode : int { LM_MASS = 0, LM_STIFF = 1, LM_DERIV = 2, LM_PIVOT = 3 };

// One array's line solve inside a launch (blockIdx.y selects the job).
template <typename T>
struct LineJob {
  const T* src;   // right-hand side (MASS, STIFF) or the differentiated field (DERIV)
  T* dst;         // result (may alias src); DERIV adds into it; PIVOT writes 1/pivot
  const T* aux;   // c (STIFF, PIVOT)
  const T* aux2;  // STIFF: inverse pivots of M + c S from an LM_PIVOT pass
  T scale;        // DERIV: dst += scale * M^-1 A src
  int dirichlet;  // 1: first and last coefficient are fixed to zero
  T* work;        // DERIV along y / z: the forward sweep's intermediate (an array in the state layout)
  // PIVOT: also store the row factors of M + c S for the streaming stiffness solve
  // (fac[m-1] = multiplier of row k-m, fac[P+e-1] = upper factor e / pivot), or NULL
  T* fac[2 * kMaxP];
};
template <typename T>
struct LineJobs {
  LineJob<T> job[3];
};

// ----------------------------------------------------------- the handle
struct Launch {  // profiling record of one kernel launch
  const char* name;
  double bytes;
  cudaEvent_t a, b;
};

struct Ctx {
  int n[3] = {0, 0, 0};  // elements x, y, z
  int N[3] = {0, 0, 0};  // coefficients per axis
  int p = 2;
  int precision = ADI_PREC_FP32;  // FP32 and MIXED keep FP32 state (element type float)
  int mixed_refine = 0;           // MIXED: one residual refinement per E half step
  int mixed_fp64_residual = 0;    // MIXED: the residual in FP64 arithmetic (default: float-float on the FP32 pipe)
  int rhs_quad = 0;               // 1: per-element material inside the right-hand side integrals (ADI_RHS_QUAD)
  void* tabq = nullptr;           // rhs_quad: element blocks of the 1D matrices per axis (element type T)
  int use_graph = 1;
  int line_tile = 0;  // lines per line-solve CTA (0: largest that leaves two CTAs per SM)
  bool line_stream = true;  // y / z stiffness solves on the streaming kernel (precomputed factors)
  bool line_xw = true;      // FP32 x mass / derivative solves on the warp-per-32-lines kernel
  double dt = 0.0;
  size_t Nc = 0;      // coefficients per component (N_x N_y N_z)
  int pitch = 0;      // device row pitch in elements: N_x rounded up to a multiple of 4
  size_t Np = 0;      // device elements per component (pitch N_y N_z)
  size_t esize = 4;
  bool factored = false;
  std::string err;

  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // the three component chains of a half step run on these streams, forked from
  // and joined back to `stream` (serial while profiling or with serial_chains)
  cudaStream_t branch[3] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[3] = {};
  int serial_chains = 0;
  int device = 0;
  int smem_optin = 48 * 1024;  // per-block opt-in shared memory (set by adi_factor)

  // per-element material (device, double), kept for set_dt
  double* d_eps = nullptr;
  double* d_mu = nullptr;
  double* d_sigma = nullptr;
  double min_eps_mu = 1.0;
  bool mu_uniform = false;  // all per-element mu equal: H half steps use 1D derivatives
  double mu_value = 1.0;
  double d_uniform = 0.0;   // tau / (2 mu) when mu_uniform

  // state and work (element type T = float or double), each Nc elements
  void* cur[6] = {};
  void* half[6] = {};  // [0..2]: E^{n+1/2}; [3..5] unused (H is updated in place)
  void* rhs[3] = {};
  void* coef[4] = {};   // a, b, c, d
  void* stage = nullptr;  // Nc doubles for host transfers (FP32 mode)
  void* pivots[3] = {};   // inverse pivots of the row-scaled M + c S, per stiffness axis
  // LU factors of the row-scaled M + c S along y and z ([axis][m]: P multipliers,
  // then P normalised upper factors), computed with the pivots; the streaming
  // y / z stiffness solves read them instead of refactoring every step
  void* stiff_fac[3][2 * kMaxP] = {};

  // 1D tables on device (element type T)
  void* tab = nullptr;
  size_t tab_bytes = 0;
  double* tab64 = nullptr;  // MIXED: the band tables in FP64 for the residual
  float2* tabff = nullptr;  // MIXED: the same tables as float pairs (hi, lo) for the float-float residual
  size_t tab64_bytes = 0;
  Axis1D axes[3];
  LuConst luconst[3][2];  // per axis: full and Dirichlet-reduced mass LU
  double* d_clock_t0 = nullptr;
  long long* d_clock_step = nullptr;
  double t_host = 0.0;
  long long steps_host = 0;

  // source
  int src_comp = -1;
  int src_i0[3] = {0, 0, 0};
  double src_w[3][kMaxP + 1] = {};
  double src_amp = 0, src_f0 = 0, src_t0 = 0, src_s = 1;

  // TMA descriptors of the state arrays (E RHS tiles), built by adi_factor
  CUtensorMap tmap_cur[6];
  CUtensorMap tmap_half[3];
  bool tmaps_ok = false;
  int* d_err = nullptr;  // device status word written by bounded waits
  int* d_bad = nullptr;  // device flag: a value that is not finite (field checks)
  // asynchronous host transfers (adi_set_fields_async / adi_fields_async): dense
  // device copies of a host state in the host's element type (in_stage, out_stage:
  // stage_bytes each, allocated by the first such call), moved over the host link by
  // the copy engines on an input and an output stream while the main stream steps;
  // events: in_stage filled / read by its commit, out_stage filled / copied out;
  // flags [0] this set's values not finite, [1] a set was refused, [2] a read saw a
  // value that is not finite (both reported by adi_sync)
  cudaStream_t io_in = nullptr, io_out = nullptr;
  void* in_stage = nullptr;
  void* out_stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t ev_in_ready = nullptr, ev_in_free = nullptr, ev_out_ready = nullptr, ev_out_free = nullptr;
  int* d_async = nullptr;
  double* d_diag = nullptr;  // 8 doubles: sums of the norm diagnostics

  // graph of one step
  cudaGraphExec_t graph = nullptr;

  // profiling
  bool profiling = false;
  std::vector<Launch*> pending;
  std::vector<adi_kernel_stat> stats;
};

// Kernel-side entry points (adi_kernels.cu), all asynchronous on ctx.stream.
cudaError_t upload_tables(Ctx& c);
cudaError_t compute_coefficients(Ctx& c);
// which 0..3: E half 1, H half 1, E half 2, H half 2; 4, 5: half step 1 or 2 (E then H)
cudaError_t run_substep(Ctx& c, int which);
// one time step (run_substep 4 then 5): the same arrays, bit for bit, as 0..3 in turn
cudaError_t run_step(Ctx& c);
// S = double or float: the element type of the dense 6 N_c layout on the host side
template <typename S>
cudaError_t set_fields_dev(Ctx& c, const S* d_src);
// convert 6 N_c values at d_src (device memory or mapped host memory) into the six
// arrays dst (state layout, constrained coefficients zero); d_bad (optional) |= 1 on NaN/Inf
template <typename S>
cudaError_t set_fields_into(Ctx& c, const S* d_src, void* const* dst, int* d_bad);
template <typename S>
cudaError_t get_fields_dev(Ctx& c, S* d_dst, int* d_bad);
// d_bad |= 1 if any of the n values at d_src is NaN or Inf
template <typename S>
cudaError_t check_finite_dev(Ctx& c, const S* d_src, long long n, int* d_bad);
cudaError_t set_clock(Ctx& c, double t0);
// copy the six scratch arrays (rhs, half) into the state and set the clock to t,
// unless *bad is set (then *refused |= 1); on c.stream
cudaError_t commit_fields(Ctx& c, const int* bad, int* refused, double t);
// squared-norm sums of the state into d_acc[6] (zeroed first):
// [int |E|^2, int |H|^2, int |grad E|^2, int |grad H|^2, int |curl E|^2, int |curl H|^2]
cudaError_t field_norms_dev(Ctx& c, double* d_acc);
// component comp on a plane grid; d_tab: 1D point records (first index, p+1 values)
cudaError_t plane_dev(Ctx& c, int comp, int axis, int nu, int nv, const double* d_tab, double* d_out);
// one bounded wait (0: E right-hand side tile wait, 1: x line bulk-copy wait) on a
// barrier that never completes, with an iteration budget; gives up into c.d_err
cudaError_t wait_selftest(Ctx& c, int which, int budget);
cudaError_t make_tensor_maps(Ctx& c);

// record a failure that has no handle (readable through adi_last_error(NULL))
adi_status fail_global(adi_status s, const std::string& msg);

// profiling hooks used by the launchers
void prof_begin(Ctx& c, const char* name, double bytes);
void prof_end(Ctx& c);

}  // namespace adi

// The opaque handle type of the C-ABI is the context itself.
struct adi_ctx : public adi::Ctx {};
