// C-ABI of the ADI isogeometric Maxwell stepper (see include/adi_maxwell.h).
// Host-side validation, ownership of device memory, CUDA-graph capture of one
// time step, and per-kernel event timing.  All arithmetic of the step runs in
// the kernels of adi_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "adi_internal.h"

using adi::Ctx;

namespace {

thread_local std::string g_create_error = "no error";

adi_status fail(Ctx* c, adi_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

adi_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? ADI_ENOMEM : ADI_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

void free_ctx(Ctx* c0) {
  if (!c0) return;
  adi_ctx* c = static_cast<adi_ctx*>(c0);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (auto* l : c->pending) delete l;
  void* ptrs[] = {c->d_eps,        c->d_mu,  c->d_sigma, c->stage,  c->tab,   c->tab64, c->tabff, c->tabq,
                  c->d_clock_t0,   c->d_clock_step, c->d_err, c->d_bad, c->d_diag, c->d_async,
                  c->in_stage,     c->out_stage};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < 6; ++i) {
    if (c->cur[i]) cudaFree(c->cur[i]);
    if (c->half[i]) cudaFree(c->half[i]);
  }
  for (int i = 0; i < 3; ++i)
    if (c->rhs[i]) cudaFree(c->rhs[i]);
  for (int i = 0; i < 4; ++i)
    if (c->coef[i]) cudaFree(c->coef[i]);
  for (int i = 0; i < 3; ++i) {
    if (c->pivots[i]) cudaFree(c->pivots[i]);
    for (int m = 0; m < 2 * adi::kMaxP; ++m)
      if (c->stiff_fac[i][m]) cudaFree(c->stiff_fac[i][m]);
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  for (cudaStream_t st : {c->io_in, c->io_out})
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : {c->ev_in_ready, c->ev_in_free, c->ev_out_ready, c->ev_out_free})
    if (ev) cudaEventDestroy(ev);
  for (int i = 0; i < 3; ++i) {
    if (c->branch[i]) cudaStreamDestroy(c->branch[i]);
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
}

// Device address of a page-locked (pinned or registered) host buffer, else null:
// kernels then read or write the caller's array directly over the host link
// instead of staging it through a copy.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

void drop_graph(Ctx* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
}

}  // namespace

// ------------------------------------------------------------- profiling
namespace adi {

adi_status fail_global(adi_status s, const std::string& msg) { return fail(nullptr, s, msg); }

void prof_begin(Ctx& c, const char* name, double bytes) {
  if (!c.profiling) return;
  Launch* l = new (std::nothrow) Launch{name, bytes, nullptr, nullptr};
  if (!l) return;
  cudaEventCreate(&l->a);
  cudaEventCreate(&l->b);
  cudaEventRecord(l->a, c.stream);
  c.pending.push_back(l);
}

void prof_end(Ctx& c) {
  if (!c.profiling || c.pending.empty()) return;
  cudaEventRecord(c.pending.back()->b, c.stream);
}

static void prof_collect(Ctx& c) {
  cudaStreamSynchronize(c.stream);
  for (Launch* l : c.pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, l->a, l->b);
    bool found = false;
    for (auto& s : c.stats)
      if (std::strcmp(s.name, l->name) == 0) {
        s.launches += 1;
        s.total_ms += ms;
        found = true;
        break;
      }
    if (!found) c.stats.push_back(adi_kernel_stat{l->name, 1, (double)ms, l->bytes});
    cudaEventDestroy(l->a);
    cudaEventDestroy(l->b);
    delete l;
  }
  c.pending.clear();
}

}  // namespace adi

// ------------------------------------------------------------------- API
extern "C" {

const char* adi_status_string(adi_status s) {
  switch (s) {
    case ADI_OK: return "ADI_OK";
    case ADI_EINVAL: return "ADI_EINVAL";
    case ADI_ENOMEM: return "ADI_ENOMEM";
    case ADI_ECUDA: return "ADI_ECUDA";
    case ADI_ESTATE: return "ADI_ESTATE";
    case ADI_ENUMERIC: return "ADI_ENUMERIC";
    case ADI_ETIMEOUT: return "ADI_ETIMEOUT";
  }
  return "ADI_UNKNOWN";
}

const char* adi_last_error(adi_handle h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

static adi_status create_impl(int nx, int ny, int nz, int p, double dt, const double* const* breaks,
                              const double* eps, const double* mu, const double* sigma, const adi_options* opt,
                              adi_handle* out);

adi_status adi_create_knots(int nx, int ny, int nz, int p, double dt, const double* breaks_x,
                            const double* breaks_y, const double* breaks_z, const double* eps, const double* mu,
                            const double* sigma, const adi_options* opt, adi_handle* out) {
  // no exception crosses the C-ABI: a failed host allocation is ADI_ENOMEM
  const double* br[3] = {breaks_x, breaks_y, breaks_z};
  try {
    return create_impl(nx, ny, nz, p, dt, br, eps, mu, sigma, opt, out);
  } catch (const std::bad_alloc&) {
    if (out) *out = nullptr;
    return fail(nullptr, ADI_ENOMEM, "adi_create: host allocation failed");
  }
}

adi_status adi_create(int nx, int ny, int nz, int p, double dt, const double* eps, const double* mu,
                      const double* sigma, const adi_options* opt, adi_handle* out) {
  return adi_create_knots(nx, ny, nz, p, dt, nullptr, nullptr, nullptr, eps, mu, sigma, opt, out);
}

// n + 1 element boundaries strictly increasing from 0 to 1
static bool breaks_ok(const double* b, int n) {
  bool ok = b[0] == 0.0 && b[n] == 1.0;
  for (int i = 0; i < n && ok; ++i) ok = std::isfinite(b[i + 1]) && b[i + 1] > b[i];
  return ok;
}

static adi_status create_impl(int nx, int ny, int nz, int p, double dt, const double* const* breaks,
                              const double* eps, const double* mu, const double* sigma, const adi_options* opt,
                              adi_handle* out) {
  if (!out) return fail(nullptr, ADI_EINVAL, "adi_create: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, ADI_EINVAL, "adi_create: element counts must be >= 1");
  const int ns[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d)
    if (breaks[d] && !breaks_ok(breaks[d], ns[d]))
      return fail(nullptr, ADI_EINVAL,
                  "adi_create_knots: element boundaries must increase strictly from 0 to 1 (n_d + 1 values)");
  if (p < 1 || p > adi::kMaxP) return fail(nullptr, ADI_EINVAL, "adi_create: p must be in 1..4");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, ADI_EINVAL, "adi_create: dt must be finite and > 0");
  int prec = ADI_PREC_FP32, use_graph = 1, refine = 1, res64 = 0, quad = 0, serial = 0;
  if (opt) {
    if (opt->precision != ADI_PREC_FP32 && opt->precision != ADI_PREC_FP64 && opt->precision != ADI_PREC_MIXED)
      return fail(nullptr, ADI_EINVAL, "adi_create: precision must be ADI_PREC_FP32, ADI_PREC_FP64 or ADI_PREC_MIXED");
    for (int i = 0; i < 2; ++i)
      if (opt->reserved[i] != 0) return fail(nullptr, ADI_EINVAL, "adi_create: reserved option fields must be 0");
    if (opt->serial_chains != 0 && opt->serial_chains != 1)
      return fail(nullptr, ADI_EINVAL, "adi_create: serial_chains must be 0 or 1");
    if (opt->rhs_material != ADI_RHS_ROW && opt->rhs_material != ADI_RHS_QUAD)
      return fail(nullptr, ADI_EINVAL, "adi_create: rhs_material must be ADI_RHS_ROW or ADI_RHS_QUAD");
    if (opt->rhs_material == ADI_RHS_QUAD && opt->precision == ADI_PREC_MIXED)
      return fail(nullptr, ADI_EINVAL, "adi_create: ADI_RHS_QUAD is not available with ADI_PREC_MIXED");
    if (opt->rhs_material == ADI_RHS_QUAD && opt->precision == ADI_PREC_FP64 && p > 3)
      return fail(nullptr, ADI_EINVAL, "adi_create: ADI_RHS_QUAD in FP64 needs p <= 3");
    if (opt->mixed_no_refine != 0 && opt->mixed_no_refine != 1)
      return fail(nullptr, ADI_EINVAL, "adi_create: mixed_no_refine must be 0 or 1");
    if (opt->mixed_fp64_residual != 0 && opt->mixed_fp64_residual != 1)
      return fail(nullptr, ADI_EINVAL, "adi_create: mixed_fp64_residual must be 0 or 1");
    prec = opt->precision;
    use_graph = opt->use_graph ? 1 : 0;
    refine = opt->mixed_no_refine ? 0 : 1;
    res64 = opt->mixed_fp64_residual;
    quad = opt->rhs_material == ADI_RHS_QUAD ? 1 : 0;
    serial = opt->serial_chains;
  }
  const size_t ne = (size_t)nx * ny * nz;
  for (const double* arr : {eps, mu}) {
    if (!arr) continue;
    for (size_t i = 0; i < ne; ++i)
      if (!(arr[i] > 0.0) || !std::isfinite(arr[i]))
        return fail(nullptr, ADI_EINVAL, "adi_create: eps and mu must be finite and > 0");
  }
  if (sigma)
    for (size_t i = 0; i < ne; ++i)
      if (!(sigma[i] >= 0.0) || !std::isfinite(sigma[i]))
        return fail(nullptr, ADI_EINVAL, "adi_create: sigma must be finite and >= 0");

  adi_ctx* c = new (std::nothrow) adi_ctx();
  if (!c) return fail(nullptr, ADI_ENOMEM, "adi_create: host allocation failed");
  c->n[0] = nx;
  c->n[1] = ny;
  c->n[2] = nz;
  c->p = p;
  for (int d = 0; d < 3; ++d) c->N[d] = c->n[d] + p;
  c->Nc = (size_t)c->N[0] * c->N[1] * c->N[2];
  c->pitch = (c->N[0] + 3) & ~3;  // 16-byte aligned rows (TMA strides) in FP32 and FP64
  c->Np = (size_t)c->pitch * c->N[1] * c->N[2];
  c->precision = prec;
  c->use_graph = use_graph;
  c->mixed_refine = prec == ADI_PREC_MIXED ? refine : 0;
  c->mixed_fp64_residual = res64;
  c->rhs_quad = quad;
  c->serial_chains = serial;
  c->esize = prec == ADI_PREC_FP64 ? 8 : 4;
  c->dt = dt;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(nullptr, e, "adi_create: cudaGetDevice");
  }
  e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(nullptr, e, "adi_create: cudaStreamCreate");
  }
  c->own_stream = true;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&c->branch[i], cudaStreamNonBlocking);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->io_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->io_out, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&c->ev_in_ready, &c->ev_in_free, &c->ev_out_ready, &c->ev_out_free})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(nullptr, e, "adi_create: branch streams");
  }
  const size_t fb = c->Np * c->esize;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  for (int i = 0; i < 6; ++i) alloc(&c->cur[i], fb);
  for (int i = 0; i < 3; ++i) alloc(&c->half[i], fb);  // E^{n+1/2}; H is updated in place
  for (int i = 0; i < 3; ++i) alloc(&c->rhs[i], fb);
  for (int i = 0; i < 4; ++i) alloc(&c->coef[i], fb);
  alloc(&c->stage, c->Nc * 6 * sizeof(double));
  alloc((void**)&c->d_eps, ne * sizeof(double));
  alloc((void**)&c->d_mu, ne * sizeof(double));
  alloc((void**)&c->d_sigma, ne * sizeof(double));
  alloc((void**)&c->d_clock_t0, sizeof(double));
  alloc((void**)&c->d_clock_step, sizeof(long long));
  alloc((void**)&c->d_err, sizeof(int));
  alloc((void**)&c->d_bad, sizeof(int));
  alloc((void**)&c->d_async, 4 * sizeof(int));
  alloc((void**)&c->d_diag, 8 * sizeof(double));
  if (!ok) {
    cudaGetLastError();
    free_ctx(c);
    return fail(nullptr, ADI_ENOMEM, "adi_create: device allocation failed");
  }
  // material: NULL -> 1, 1, 0
  std::vector<double> tmp;
  try {
    tmp.resize(ne);
  } catch (const std::bad_alloc&) {
    free_ctx(c);
    return fail(nullptr, ADI_ENOMEM, "adi_create: host allocation failed");
  }
  const double* srcs[3] = {eps, mu, sigma};
  double* dsts[3] = {c->d_eps, c->d_mu, c->d_sigma};
  const double defaults[3] = {1.0, 1.0, 0.0};
  for (int k = 0; k < 3; ++k) {
    const double* s = srcs[k];
    if (!s) {
      std::fill(tmp.begin(), tmp.end(), defaults[k]);
      s = tmp.data();
    }
    e = cudaMemcpy(dsts[k], s, ne * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_ctx(c);
      return cuda_fail(nullptr, e, "adi_create: upload material");
    }
  }
  c->mu_uniform = true;
  c->mu_value = mu ? mu[0] : 1.0;
  if (mu)
    for (size_t i = 1; i < ne; ++i)
      if (mu[i] != mu[0]) {
        c->mu_uniform = false;
        break;
      }
  c->d_uniform = dt / (2.0 * c->mu_value);
  for (int d = 0; d < 3; ++d) adi::build_axis(c->n[d], p, c->axes[d], breaks[d]);
  e = adi::compute_coefficients(*c);
  if (e == cudaSuccess) {
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
      e = cudaMemsetAsync(c->cur[i], 0, fb, c->stream);
      if (e == cudaSuccess && i < 3) e = cudaMemsetAsync(c->half[i], 0, fb, c->stream);
    }
  }
  if (e == cudaSuccess) e = adi::set_clock(*c, 0.0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_async, 0, 4 * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(nullptr, e, "adi_create: setup kernels");
  }
  c->err = "no error";
  *out = c;
  return ADI_OK;
}

// shared checks and axis construction of the host-only axis calls
static adi_status host_axis(int n, int p, const double* breaks, const char* name, adi::Axis1D& ax) {
  if (n < 1) return fail(nullptr, ADI_EINVAL, std::string(name) + ": n must be >= 1");
  if (p < 1 || p > adi::kMaxP) return fail(nullptr, ADI_EINVAL, std::string(name) + ": p must be in 1..4");
  if (breaks && !breaks_ok(breaks, n))
    return fail(nullptr, ADI_EINVAL,
                std::string(name) + ": element boundaries must increase strictly from 0 to 1 (n + 1 values)");
  try {
    adi::build_axis(n, p, ax, breaks);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, ADI_ENOMEM, std::string(name) + ": host allocation failed");
  }
  return ADI_OK;
}

adi_status adi_axis_bands(int n, int p, const double* breaks, double* M, double* S, double* A, double* B,
                          int* inner) {
  adi::Axis1D ax;
  adi_status st = host_axis(n, p, breaks, "adi_axis_bands", ax);
  if (st != ADI_OK) return st;
  double* outs[4] = {M, S, A, B};
  const std::vector<double>* src[4] = {&ax.M, &ax.S, &ax.A, &ax.B};
  for (int o = 0; o < 4; ++o)
    if (outs[o]) std::copy(src[o]->begin(), src[o]->end(), outs[o]);
  if (inner) {
    inner[0] = ax.inner_lo;
    inner[1] = ax.inner_hi;
  }
  return ADI_OK;
}

adi_status adi_axis_tables(int n, int p, const double* breaks, double* G, double* lam) {
  adi::Axis1D ax;
  adi_status st = host_axis(n, p, breaks, "adi_axis_tables", ax);
  if (st != ADI_OK) return st;
  if (G) std::copy(ax.G.begin(), ax.G.end(), G);
  if (lam) {
    try {
      *lam = adi::lambda_max(ax);
    } catch (const std::bad_alloc&) {
      return fail(nullptr, ADI_ENOMEM, "adi_axis_tables: host allocation failed");
    }
  }
  return ADI_OK;
}

adi_status adi_axis_element_matrices(int n, int p, const double* breaks, double* loc) {
  if (!loc) return fail(nullptr, ADI_EINVAL, "adi_axis_element_matrices: NULL output");
  adi::Axis1D ax;
  adi_status st = host_axis(n, p, breaks, "adi_axis_element_matrices", ax);
  if (st != ADI_OK) return st;
  std::vector<double> blocks;
  try {
    adi::element_matrices(ax, blocks);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, ADI_ENOMEM, "adi_axis_element_matrices: host allocation failed");
  }
  std::copy(blocks.begin(), blocks.end(), loc);
  return ADI_OK;
}

adi_status adi_axis_mass_lu(int n, int p, const double* breaks, int reduced, double* L, double* inv_d, double* U) {
  if (reduced != 0 && reduced != 1) return fail(nullptr, ADI_EINVAL, "adi_axis_mass_lu: reduced must be 0 or 1");
  if (!L || !inv_d || !U) return fail(nullptr, ADI_EINVAL, "adi_axis_mass_lu: NULL output");
  adi::Axis1D ax;
  adi_status st = host_axis(n, p, breaks, "adi_axis_mass_lu", ax);
  if (st != ADI_OK) return st;
  adi::BandLU lu;
  try {
    adi::band_lu(ax.M, nullptr, ax.N, p, reduced ? 1 : 0, reduced ? ax.N - 2 : ax.N - 1, lu);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, ADI_ENOMEM, "adi_axis_mass_lu: host allocation failed");
  }
  std::copy(lu.L.begin(), lu.L.end(), L);
  std::copy(lu.inv_d.begin(), lu.inv_d.end(), inv_d);
  std::copy(lu.U.begin(), lu.U.end(), U);
  return ADI_OK;
}

adi_status adi_axis_point_basis(int n, int p, const double* breaks, double x0, int* first, double* vals) {
  if (!(x0 >= 0.0 && x0 <= 1.0)) return fail(nullptr, ADI_EINVAL, "adi_axis_point_basis: x0 must lie in [0,1]");
  if (!first || !vals) return fail(nullptr, ADI_EINVAL, "adi_axis_point_basis: NULL output");
  adi::Axis1D ax;
  adi_status st = host_axis(n, p, breaks, "adi_axis_point_basis", ax);
  if (st != ADI_OK) return st;
  *first = adi::point_basis(ax, x0, vals);
  return ADI_OK;
}

adi_status adi_factor(adi_handle h) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_factor: NULL handle");
  cudaError_t e = adi::upload_tables(*h);
  if (e == cudaSuccess) e = adi::make_tensor_maps(*h);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_factor");
  drop_graph(h);
  h->factored = true;
  return ADI_OK;
}

adi_status adi_set_dt(adi_handle h, double dt) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_set_dt: NULL handle");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, ADI_EINVAL, "adi_set_dt: dt must be finite and > 0");
  h->dt = dt;
  h->d_uniform = dt / (2.0 * h->mu_value);
  cudaError_t e = adi::compute_coefficients(*h);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_set_dt");
  drop_graph(h);
  h->factored = false;
  return ADI_OK;
}

adi_status adi_set_stream(adi_handle h, void* s) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_set_stream: NULL handle");
  cudaError_t e = cudaStreamSynchronize(h->stream);  // (its waits cover pending asynchronous transfers)
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->io_in);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->io_out);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_set_stream");
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->own_stream = false;
  h->stream = (cudaStream_t)s;
  drop_graph(h);
  return ADI_OK;
}

}  // extern "C"

extern "C" {
static adi_status check_device_status(adi_handle h, const char* where);
}

// Shared by adi_set_fields (S = double) and adi_set_fields_f32 (S = float).
template <typename S>
static adi_status set_fields_impl(adi_handle h, const S* EH, double t, const char* name) {
  if (!h) return fail(nullptr, ADI_EINVAL, std::string(name) + ": NULL handle");
  if (!EH) return fail(h, ADI_EINVAL, std::string(name) + ": EH is NULL");
  if (reinterpret_cast<uintptr_t>(EH) % sizeof(S) != 0)
    return fail(h, ADI_EINVAL, std::string(name) + ": EH is not aligned to its element size");
  if (!std::isfinite(t)) return fail(h, ADI_EINVAL, std::string(name) + ": t must be finite");
  // check on the device (a host scan of 6 N_c values would dominate the call); the
  // state is written only when every value is finite.  A page-locked EH is converted
  // in one pass straight from host memory into scratch arrays (the right-hand side
  // and half-step buffers, free between steps; a partial step is discarded), then
  // copied into the state; other memory is copied to the staging buffer first.
  const long long n6 = 6LL * (long long)h->Nc;
  const S* mapped = static_cast<const S*>(mapped_host(EH));
  void* scratch[6] = {h->rhs[0], h->rhs[1], h->rhs[2], h->half[0], h->half[1], h->half[2]};
  cudaError_t e = cudaMemsetAsync(h->d_bad, 0, sizeof(int), h->stream);
  if (mapped) {
    if (e == cudaSuccess) e = adi::set_fields_into<S>(*h, mapped, scratch, h->d_bad);
  } else {
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->stage, EH, n6 * sizeof(S), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = adi::check_finite_dev<S>(*h, (const S*)h->stage, n6, h->d_bad);
  }
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, h->d_bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, name);
  if (bad) return fail(h, ADI_ENUMERIC, std::string(name) + ": NaN or Inf in EH");
  if (mapped) {
    for (int i = 0; i < 6 && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(h->cur[i], scratch[i], h->Np * h->esize, cudaMemcpyDeviceToDevice, h->stream);
  } else {
    e = adi::set_fields_dev<S>(*h, (const S*)h->stage);
  }
  if (e == cudaSuccess) e = adi::set_clock(*h, t);
  if (e != cudaSuccess) return cuda_fail(h, e, name);
  h->t_host = t;
  h->steps_host = 0;
  return ADI_OK;
}

// Shared by adi_fields (S = double) and adi_fields_f32 (S = float).
template <typename S>
static adi_status fields_impl(adi_handle h, S* EH, double* t, const char* name) {
  if (!h) return fail(nullptr, ADI_EINVAL, std::string(name) + ": NULL handle");
  if (!EH) return fail(h, ADI_EINVAL, std::string(name) + ": EH is NULL");
  if (reinterpret_cast<uintptr_t>(EH) % sizeof(S) != 0)
    return fail(h, ADI_EINVAL, std::string(name) + ": EH is not aligned to its element size");
  // a page-locked EH is written directly by the kernel, other memory through the staging buffer
  S* mapped = const_cast<S*>(static_cast<const S*>(mapped_host(EH)));
  cudaError_t e = cudaMemsetAsync(h->d_bad, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = adi::get_fields_dev<S>(*h, mapped ? mapped : (S*)h->stage, h->d_bad);
  if (e == cudaSuccess && !mapped)
    e = cudaMemcpyAsync(EH, h->stage, 6 * h->Nc * sizeof(S), cudaMemcpyDeviceToHost, h->stream);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, h->d_bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, name);
  if (t) *t = h->t_host + (double)h->steps_host * h->dt;
  adi_status ds = check_device_status(h, name);
  if (ds != ADI_OK) return ds;
  if (bad) return fail(h, ADI_ENUMERIC, std::string(name) + ": NaN or Inf in the state");
  return ADI_OK;
}

extern "C" {

adi_status adi_set_fields(adi_handle h, const double* EH, double t) {
  return set_fields_impl<double>(h, EH, t, "adi_set_fields");
}

adi_status adi_set_fields_f32(adi_handle h, const float* EH, double t) {
  return set_fields_impl<float>(h, EH, t, "adi_set_fields_f32");
}

adi_status adi_set_source(adi_handle h, double x0, double y0, double z0, int comp, double amp, double f0,
                          double t0, double s) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_set_source: NULL handle");
  const double xs[3] = {x0, y0, z0};
  for (double v : xs)
    if (!(v >= 0.0 && v <= 1.0)) return fail(h, ADI_EINVAL, "adi_set_source: position must lie in [0,1]^3");
  if (comp < 0 || comp > 2) return fail(h, ADI_EINVAL, "adi_set_source: comp must be 0, 1 or 2");
  if (!std::isfinite(amp) || !std::isfinite(f0) || !std::isfinite(t0) || !(s > 0.0) || !std::isfinite(s))
    return fail(h, ADI_EINVAL, "adi_set_source: amp, f0, t0 must be finite and s > 0");
  for (int d = 0; d < 3; ++d) {
    double v[adi::kMaxP + 1] = {};
    h->src_i0[d] = adi::point_basis(h->axes[d], xs[d], v);
    for (int q = 0; q <= adi::kMaxP; ++q) h->src_w[d][q] = q <= h->p ? v[q] : 0.0;
  }
  h->src_comp = comp;
  h->src_amp = amp;
  h->src_f0 = f0;
  h->src_t0 = t0;
  h->src_s = s;
  drop_graph(h);
  return ADI_OK;
}

static adi_status capture_graph(adi_handle h) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_step: begin capture");
  cudaError_t ek = cudaSuccess;
  ek = adi::run_step(*h);
  e = cudaStreamEndCapture(h->stream, &g);
  if (ek != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, ek, "adi_step: kernel launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_step: end capture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return cuda_fail(h, e, "adi_step: instantiate");
  }
  return ADI_OK;
}

adi_status adi_step(adi_handle h, int n) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_step: NULL handle");
  if (n < 1) return fail(h, ADI_EINVAL, "adi_step: n must be >= 1");
  if (!h->factored) return fail(h, ADI_ESTATE, "adi_step: call adi_factor first");
  const bool graph = h->use_graph && !h->profiling && h->stream != nullptr;
  if (graph && !h->graph) {
    adi_status s = capture_graph(h);
    if (s != ADI_OK) return s;
  }
  for (int k = 0; k < n; ++k) {
    cudaError_t e = cudaSuccess;
    if (graph) {
      e = cudaGraphLaunch(h->graph, h->stream);
    } else {
      e = adi::run_step(*h);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "adi_step");
    h->steps_host += 1;
  }
  return ADI_OK;
}

adi_status adi_substep(adi_handle h, int which) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_substep: NULL handle");
  if (which < 0 || which > 3) return fail(h, ADI_EINVAL, "adi_substep: which must be 0..3");
  if (!h->factored) return fail(h, ADI_ESTATE, "adi_substep: call adi_factor first");
  cudaError_t e = adi::run_substep(*h, which);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_substep");
  if (which == 3) h->steps_host += 1;
  return ADI_OK;
}

// Read and clear the device status word: a bounded wait that gave up is
// reported once, by the first call that synchronises after it.
static adi_status check_device_status(adi_handle h, const char* where) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  if (err) {
    e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, where);
    return fail(h, ADI_ETIMEOUT, std::string(where) + ": a bounded device wait gave up (TMA tile not delivered)");
  }
  return ADI_OK;
}

adi_status adi_wait_selftest(adi_handle h, int which, int budget) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_wait_selftest: NULL handle");
  if (which < 0 || which > 1) return fail(h, ADI_EINVAL, "adi_wait_selftest: which must be 0 or 1");
  if (budget < 0 || budget > (1 << 22)) return fail(h, ADI_EINVAL, "adi_wait_selftest: budget must be in 0..2^22");
  cudaError_t e = adi::wait_selftest(*h, which, budget);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_wait_selftest");
  return ADI_OK;
}

adi_status adi_fields(adi_handle h, double* EH, double* t) { return fields_impl<double>(h, EH, t, "adi_fields"); }

adi_status adi_fields_f32(adi_handle h, float* EH, double* t) { return fields_impl<float>(h, EH, t, "adi_fields_f32"); }

adi_status adi_fields_device(adi_handle h, void* dev_ptr, void* stream) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_fields_device: NULL handle");
  if (!dev_ptr) return fail(h, ADI_EINVAL, "adi_fields_device: dev_ptr is NULL");
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  const size_t fb = h->Nc * h->esize;  // dense output, N_x elements per row
  if (s != h->stream) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "adi_fields_device");
  }
  for (int i = 0; i < 6; ++i) {
    cudaError_t e = cudaMemcpy2DAsync((char*)dev_ptr + i * fb, h->N[0] * h->esize, h->cur[i], h->pitch * h->esize,
                                      h->N[0] * h->esize, (size_t)h->N[1] * h->N[2], cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "adi_fields_device");
  }
  return ADI_OK;
}

adi_status adi_norms(adi_handle h, double* out) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_norms: NULL handle");
  if (!out) return fail(h, ADI_EINVAL, "adi_norms: out is NULL");
  double acc[6] = {};
  cudaError_t e = adi::field_norms_dev(*h, h->d_diag);
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, h->d_diag, sizeof(acc), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_norms");
  // rounding can leave a tiny negative sum for a zero field
  for (double& v : acc) v = v > 0.0 ? v : 0.0;
  out[0] = std::sqrt(acc[0]);
  out[1] = std::sqrt(acc[1]);
  out[2] = std::sqrt(acc[0] + acc[2]);
  out[3] = std::sqrt(acc[1] + acc[3]);
  out[4] = std::sqrt(acc[0] + acc[4]);
  out[5] = std::sqrt(acc[1] + acc[5]);
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(out[i])) return fail(h, ADI_ENUMERIC, "adi_norms: NaN or Inf in the state");
  return ADI_OK;
}

adi_status adi_plane(adi_handle h, int comp, int axis, double pos, int nu, int nv, double* out) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_plane: NULL handle");
  if (!out) return fail(h, ADI_EINVAL, "adi_plane: out is NULL");
  if (comp < 0 || comp > 5 || axis < 0 || axis > 2) return fail(h, ADI_EINVAL, "adi_plane: comp 0..5, axis 0..2");
  if (!(pos >= 0.0 && pos <= 1.0)) return fail(h, ADI_EINVAL, "adi_plane: pos must lie in [0, 1]");
  if (nu < 2 || nv < 2) return fail(h, ADI_EINVAL, "adi_plane: nu, nv must be >= 2");
  const int rec = h->p + 2;
  const long long ntab = (long long)rec * (1 + nu + nv);
  const long long nout = (long long)nu * nv;
  if (ntab + nout > 6LL * (long long)h->Nc)
    return fail(h, ADI_EINVAL, "adi_plane: nu * nv exceeds the handle's staging buffer (6 N_c doubles)");
  // 1D point records (first B-spline index, p + 1 values): the plane's coordinate, then the u and v points
  const int o0 = axis == 0 ? 1 : 0, o1 = axis == 2 ? 1 : 2;
  std::vector<double> tab((size_t)ntab, 0.0);
  auto put = [&](long long slot, int d, double x) {
    double v[adi::kMaxP + 1] = {};
    const int e = adi::point_basis(h->axes[d], x, v);
    tab[(size_t)(slot * rec)] = (double)e;
    for (int q = 0; q <= h->p; ++q) tab[(size_t)(slot * rec + 1 + q)] = v[q];
  };
  put(0, axis, pos);
  for (int j = 0; j < nu; ++j) put(1 + j, o0, (double)j / (nu - 1));
  for (int k = 0; k < nv; ++k) put(1 + nu + k, o1, (double)k / (nv - 1));
  double* d_tab = static_cast<double*>(h->stage);
  double* d_out = d_tab + ntab;
  cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), (size_t)ntab * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = adi::plane_dev(*h, comp, axis, nu, nv, d_tab, d_out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, (size_t)nout * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_plane");
  return ADI_OK;
}

double adi_cfl_dt(adi_handle h) {
  if (!h) return -1.0;
  double lam = 0.0;
  for (int d = 0; d < 3; ++d) lam += adi::lambda_max(h->axes[d]);
  if (!(lam > 0.0) || !(h->min_eps_mu > 0.0)) return -1.0;
  double cmax = 1.0 / std::sqrt(h->min_eps_mu);
  return 2.0 / (cmax * std::sqrt(lam));
}

adi_status adi_sync(adi_handle h) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_sync: NULL handle");
  cudaError_t e = cudaStreamSynchronize(h->io_in);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->io_out);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_sync");
  adi_status ds = check_device_status(h, "adi_sync");
  if (ds != ADI_OK) return ds;
  // outcomes of the asynchronous transfers since the last report (then cleared)
  int fl[4] = {0, 0, 0, 0};
  e = cudaMemcpy(fl, h->d_async, sizeof(fl), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && (fl[1] || fl[2])) e = cudaMemset(h->d_async, 0, sizeof(fl));
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_sync");
  if (fl[1]) return fail(h, ADI_ENUMERIC, "adi_sync: a field set by adi_set_fields_async held NaN or Inf and was not applied");
  if (fl[2]) return fail(h, ADI_ENUMERIC, "adi_sync: a state read by adi_fields_async holds NaN or Inf");
  return ADI_OK;
}

// Checks shared by the asynchronous transfers: EH page-locked (pinned or
// registered, so that the copy engines move it without a host-side staging copy)
// and aligned to elem_bytes = 4 or 8.
static adi_status async_host(adi_handle h, const void* EH, int elem_bytes, const char* name) {
  if (!h) return fail(nullptr, ADI_EINVAL, std::string(name) + ": NULL handle");
  if (elem_bytes != 4 && elem_bytes != 8)
    return fail(h, ADI_EINVAL, std::string(name) + ": elem_bytes must be 4 (float) or 8 (double)");
  if (!EH || reinterpret_cast<uintptr_t>(EH) % elem_bytes != 0)
    return fail(h, ADI_EINVAL, std::string(name) + ": EH is NULL or not aligned to elem_bytes");
  if (!mapped_host(EH))
    return fail(h, ADI_EINVAL, std::string(name) + ": EH must be page-locked host memory (pinned or registered)");
  return ADI_OK;
}

// The two device staging arrays, at least `bytes` each (a larger request, e.g.
// doubles after floats, replaces them once the work that uses them is done).
static adi_status async_stage(adi_handle h, size_t bytes, const char* name) {
  if (h->stage_bytes >= bytes) return ADI_OK;
  cudaError_t e = cudaStreamSynchronize(h->io_in);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->io_out);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, name);
  for (void** p : {&h->in_stage, &h->out_stage}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  h->stage_bytes = 0;
  e = cudaMalloc(&h->in_stage, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->out_stage, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (void** p : {&h->in_stage, &h->out_stage}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
    return fail(h, ADI_ENOMEM, std::string(name) + ": device staging allocation failed");
  }
  h->stage_bytes = bytes;
  return ADI_OK;
}

// Set: the copy engine moves EH into in_stage on the input stream as soon as the
// previous set's commit has read in_stage (so during the steps enqueued before
// the call); the main stream then converts it into the scratch arrays and
// commits it after everything enqueued before the call.
adi_status adi_set_fields_async(adi_handle h, const void* EH, int elem_bytes, double t) {
  adi_status st = async_host(h, EH, elem_bytes, "adi_set_fields_async");
  if (st != ADI_OK) return st;
  if (!std::isfinite(t)) return fail(h, ADI_EINVAL, "adi_set_fields_async: t must be finite");
  const size_t bytes = 6 * h->Nc * (size_t)elem_bytes;
  st = async_stage(h, bytes, "adi_set_fields_async");
  if (st != ADI_OK) return st;
  void* scratch[6] = {h->rhs[0], h->rhs[1], h->rhs[2], h->half[0], h->half[1], h->half[2]};
  cudaError_t e = cudaStreamWaitEvent(h->io_in, h->ev_in_free, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->in_stage, EH, bytes, cudaMemcpyHostToDevice, h->io_in);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_in_ready, h->io_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_in_ready, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_async, 0, sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = elem_bytes == 4 ? adi::set_fields_into<float>(*h, static_cast<const float*>(h->in_stage), scratch, h->d_async)
                        : adi::set_fields_into<double>(*h, static_cast<const double*>(h->in_stage), scratch, h->d_async);
  if (e == cudaSuccess) e = adi::commit_fields(*h, h->d_async, h->d_async + 1, t);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_in_free, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_set_fields_async");
  h->t_host = t;
  h->steps_host = 0;
  return ADI_OK;
}

// Read: the main stream converts the state into out_stage after everything
// enqueued before the call (once the previous read's copy has left out_stage);
// the copy engine then moves it to EH on the output stream while the main
// stream goes on with the work enqueued after the call.
adi_status adi_fields_async(adi_handle h, void* EH, int elem_bytes) {
  adi_status st = async_host(h, EH, elem_bytes, "adi_fields_async");
  if (st != ADI_OK) return st;
  const size_t bytes = 6 * h->Nc * (size_t)elem_bytes;
  st = async_stage(h, bytes, "adi_fields_async");
  if (st != ADI_OK) return st;
  cudaError_t e = cudaStreamWaitEvent(h->stream, h->ev_out_free, 0);
  if (e == cudaSuccess)
    e = elem_bytes == 4 ? adi::get_fields_dev<float>(*h, static_cast<float*>(h->out_stage), h->d_async + 2)
                        : adi::get_fields_dev<double>(*h, static_cast<double*>(h->out_stage), h->d_async + 2);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_out_ready, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->io_out, h->ev_out_ready, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(EH, h->out_stage, bytes, cudaMemcpyDeviceToHost, h->io_out);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_out_free, h->io_out);
  if (e != cudaSuccess) return cuda_fail(h, e, "adi_fields_async");
  return ADI_OK;
}

adi_status adi_set_profiling(adi_handle h, int on) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_set_profiling: NULL handle");
  adi::prof_collect(*h);
  h->profiling = on != 0;
  h->stats.clear();
  return ADI_OK;
}

adi_status adi_kernel_stats(adi_handle h, adi_kernel_stat* out, int max, int* count) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_kernel_stats: NULL handle");
  if (!count || (max > 0 && !out)) return fail(h, ADI_EINVAL, "adi_kernel_stats: NULL output");
  adi::prof_collect(*h);
  int n = (int)h->stats.size();
  for (int i = 0; i < n && i < max; ++i) out[i] = h->stats[i];
  *count = n;
  return ADI_OK;
}

adi_status adi_dims(adi_handle h, int* Nx, int* Ny, int* Nz, int* elem_bytes) {
  if (!h) return fail(nullptr, ADI_EINVAL, "adi_dims: NULL handle");
  if (Nx) *Nx = h->N[0];
  if (Ny) *Ny = h->N[1];
  if (Nz) *Nz = h->N[2];
  if (elem_bytes) *elem_bytes = (int)h->esize;
  return ADI_OK;
}

void adi_destroy(adi_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaStreamSynchronize(h->io_in);  // copies of the asynchronous transfers
  cudaStreamSynchronize(h->io_out);
  free_ctx(h);
}

}  // extern "C"
