// Allocation-free entry point: the explicit time-step limit from per-element
// material that the caller already holds in device memory (see
// adi_cfl_dt_noalloc in include/adi_maxwell.h).
//
// Every other call of this library either allocates device memory itself
// (adi_create, adi_fields) or needs a handle that did.  Some callers cannot
// allocate at the point where they need the time step: services that hand all
// device memory to their own pool at start-up and forbid later
// cudaMalloc/cudaFree, real-time loops that must not block in the allocator,
// and plug-ins of a host application that owns every device allocation.  They
// can call this function instead: its scratch (the 1D element-integral tables,
// the running minimum and a bad-material flag) lives in the file-scope array
// below, which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include <string>

#include "adi_internal.h"

namespace {

constexpr int kNoallocScratchDoubles = 8192;  // 64 KiB
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];
// layout: [0] running minimum (as the bits of a positive double),
//         [1] flag: nonzero when some eps or mu element is not finite and > 0,
//         [8 ..] element-integral tables of x, y, z (N_d * (p + 1) each)
constexpr int kTablesOffset = 8;

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

// Same arithmetic as the per-row material of adi_create: support-weighted
// mean of eps and mu per test function, then the minimum of eps^ * mu^.  The
// minimum is taken with atomicMin on the bit patterns, an order that holds for
// positive doubles only, so every element is checked first: any eps or mu that
// is not finite and > 0 (negative, zero, NaN, Inf) sets the flag instead, and
// so does a row product that is not finite and > 0.
__global__ void min_eps_mu_kernel(const double* __restrict__ eps, const double* __restrict__ mu,
                                  const double* __restrict__ scratch, int nx, int ny, int nz, int p,
                                  int offx, int offy, int offz, unsigned long long* min_bits,
                                  unsigned long long* bad) {
  const int Nx = nx + p, Ny = ny + p, Nz = nz + p;
  const long long Nc = (long long)Nx * Ny * Nz;
  const long long ne = (long long)nx * ny * nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  bool local_bad = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += stride) {
    const double ve = eps[e], vm = mu[e];
    if (!(ve > 0.0 && isfinite(ve)) || !(vm > 0.0 && isfinite(vm))) local_bad = true;
  }
  const double* Gx = scratch + offx;
  const double* Gy = scratch + offy;
  const double* Gz = scratch + offz;
  double local_min = 1e300;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < Nc; g += stride) {
    int r = (int)(g % Nx), s = (int)((g / Nx) % Ny), t = (int)(g / ((long long)Nx * Ny));
    double ne_ = 0, nm = 0, den = 0;
    for (int c = 0; c <= p; ++c) {
      int ez = t - p + c;
      if (ez < 0 || ez >= nz) continue;
      double wz = Gz[t * (p + 1) + c];
      for (int b = 0; b <= p; ++b) {
        int ey = s - p + b;
        if (ey < 0 || ey >= ny) continue;
        double wyz = wz * Gy[s * (p + 1) + b];
        for (int a = 0; a <= p; ++a) {
          int ex = r - p + a;
          if (ex < 0 || ex >= nx) continue;
          double w = wyz * Gx[r * (p + 1) + a];
          long long e = ((long long)ez * ny + ey) * nx + ex;
          ne_ += w * eps[e];
          nm += w * mu[e];
          den += w;
        }
      }
    }
    const double prod = (ne_ / den) * (nm / den);
    if (prod > 0.0 && isfinite(prod)) local_min = fmin(local_min, prod);
    else local_bad = true;
  }
  if (local_bad) atomicOr(bad, 1ULL);
  atomicMin(min_bits, (unsigned long long)__double_as_longlong(local_min));
}

__global__ void reset_min_kernel(unsigned long long* min_bits, unsigned long long* bad) {
  *min_bits = 0x7FEFFFFFFFFFFFFFULL;
  *bad = 0ULL;
}

}  // namespace

extern "C" adi_status adi_cfl_dt_noalloc(int nx, int ny, int nz, int p, const double* d_eps, const double* d_mu,
                                         void* cuda_stream, double* dt_out) {
  if (!dt_out || !d_eps || !d_mu) return adi::fail_global(ADI_EINVAL, "adi_cfl_dt_noalloc: NULL pointer");
  if (nx < 1 || ny < 1 || nz < 1) return adi::fail_global(ADI_EINVAL, "adi_cfl_dt_noalloc: element counts must be >= 1");
  if (p < 1 || p > adi::kMaxP) return adi::fail_global(ADI_EINVAL, "adi_cfl_dt_noalloc: p must be in 1..4");
  // widened term by term: the int sum nx + ny + nz may wrap for huge sizes
  const long long need = kTablesOffset + ((long long)nx + ny + nz + 3LL * p) * (p + 1);
  if (need > kNoallocScratchDoubles)
    return adi::fail_global(ADI_EINVAL,
                            "adi_cfl_dt_noalloc: (nx + ny + nz + 3p) * (p + 1) exceeds the 8184-double scratch limit");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return adi::fail_global(ADI_ECUDA, "adi_cfl_dt_noalloc: no usable current device");
  if (!g_scratch_ptr[dev]) {  // first call on this device: look up the array's device address
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
      return adi::fail_global(ADI_ECUDA, std::string("adi_cfl_dt_noalloc: cudaGetSymbolAddress: ") +
                                             cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(ptr);
  }
  double* scratch = g_scratch_ptr[dev];
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // host tables (FP64, no device memory), copied into the scratch
  adi::Axis1D ax[3];
  const int n[3] = {nx, ny, nz};
  std::vector<double> G;
  int off[3];
  for (int d = 0; d < 3; ++d) {
    adi::build_axis(n[d], p, ax[d]);
    off[d] = kTablesOffset + (int)G.size();
    G.insert(G.end(), ax[d].G.begin(), ax[d].G.end());
  }
  unsigned long long* min_bits = reinterpret_cast<unsigned long long*>(scratch);
  unsigned long long* bad = min_bits + 1;
  e = cudaMemcpyAsync(scratch + kTablesOffset, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    reset_min_kernel<<<1, 1, 0, s>>>(min_bits, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const long long Nc = (long long)(nx + p) * (ny + p) * (nz + p);
    long long b = (Nc + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    min_eps_mu_kernel<<<(unsigned)b, 256, 0, s>>>(d_eps, d_mu, scratch, nx, ny, nz, p, off[0], off[1], off[2], min_bits,
                                                   bad);
    e = cudaGetLastError();
  }
  unsigned long long res[2] = {0ULL, 0ULL};  // minimum bits, bad-material flag
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, min_bits, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return adi::fail_global(ADI_ECUDA, std::string("adi_cfl_dt_noalloc: ") + cudaGetErrorString(e));
  if (res[1]) return adi::fail_global(ADI_ENUMERIC, "adi_cfl_dt_noalloc: eps and mu must be finite and > 0");
  double m;
  std::memcpy(&m, &res[0], sizeof(m));
  double lam = 0.0;
  for (int d = 0; d < 3; ++d) lam += adi::lambda_max(ax[d]);
  if (!(m > 0.0) || !(lam > 0.0)) return adi::fail_global(ADI_ENUMERIC, "adi_cfl_dt_noalloc: non-positive material");
  *dt_out = 2.0 * std::sqrt(m) / std::sqrt(lam);
  return ADI_OK;
}
