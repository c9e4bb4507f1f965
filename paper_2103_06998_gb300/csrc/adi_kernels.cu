// CUDA kernels of the ADI isogeometric Maxwell step (sm_103a).
//
// One time step is four sub-solves (eqs. scheme1a-1d of the paper, discretised
// as eqs. discrete1-discrete4):
//   E half step 1: RHS (eq. dupa1ab, rows scaled by a, b, c) -> stiffness
//                  direction line solve (row-scaled M + c S) -> two mass
//                  direction line solves (Appendix, eqs. split1/split2);
//   H half step 1: RHS (eq. discrete2, rows scaled by d) -> three mass solves;
//   E half step 2: as half step 1 with K2 / R2 (eq. discrete3);
//   H half step 2: eq. discrete4 with the minus sign of eq. scheme1d on C1.
//
// Kernels:
//   rhs_kernel   sum-factorised Kronecker contractions on a 3D tile held in
//                shared memory (z pass, y pass, x pass per term), all terms of
//                one sub-step in one launch, each input tile loaded once.
//   line_kernel  banded Gaussian elimination without pivoting along x, y or z,
//                one thread per line; a tile of lines is staged in shared
//                memory (coalesced, transposed to line-major for x), solved in
//                place and written back.  STIFF=true factors the row-scaled
//                M + c S on the fly; otherwise the precomputed mass LU is used.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "adi_internal.h"

namespace adi {

namespace {

unsigned grid_for(long long n, int threads);

// Does the tile [x0, x0+tx) x [y0, y0+ty) x [z0, z0+tz) hold a coefficient of the
// point source's support i0 .. i0 + p (per axis)?  Only such tiles evaluate the
// source's time profile (sin and exp in FP64).
__device__ __forceinline__ bool src_in_tile(const int (&i0)[3], int p, int x0, int y0, int z0, int tx, int ty,
                                            int tz) {
  return i0[0] <= x0 + tx - 1 && i0[0] + p >= x0 && i0[1] <= y0 + ty - 1 && i0[1] + p >= y0 &&
         i0[2] <= z0 + tz - 1 && i0[2] + p >= z0;
}

// ------------------------------------------------------------------ RHS
template <typename T, int P, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY) rhs_kernel(const RhsParams<T> prm) {
  constexpr int W = 2 * P + 1;
  constexpr int HX = TX + 2 * P, HY = TY + 2 * P, HZ = TZ + 2 * P;
  constexpr int NT = TX * TY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_in = reinterpret_cast<T*>(smem_raw);
  T* s_z = s_in + HZ * HY * HX;
  T* s_y = s_z + TZ * HY * HX;
  __shared__ T s_bx[TX][W], s_by[TY][W], s_bz[TZ][W];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int Nx = prm.Nx, Ny = prm.Ny, Nz = prm.Nz, pitch = prm.pitch;
  const long long sxy = (long long)pitch * Ny;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool col_in = gx < Nx && gy < Ny;

  // row coefficients of this thread's outputs
  T cf[5][TZ];
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) cf[k][zz] = T(k == 0 ? 1 : 0);
#pragma unroll
  for (int k = 1; k < 5; ++k) {
    if (prm.coef[k] != nullptr && col_in) {
#pragma unroll
      for (int zz = 0; zz < TZ; ++zz) {
        int gz = z0 + zz;
        if (gz < Nz) cf[k][zz] = prm.coef[k][gz * sxy + (long long)gy * pitch + gx];
      }
    }
  }

  T acc[3][TZ];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) acc[c][zz] = T(0);

  int cur_field = -1;
  for (int t = 0; t < prm.nterms; ++t) {
    const Term tm = prm.terms[t];
    __syncthreads();  // previous x pass done with s_y / band rows
    if (tm.field != cur_field) {
      const T* __restrict__ f = prm.fields[tm.field];
      for (int i = tid; i < HZ * HY * HX; i += NT) {
        int xx = i % HX, r = i / HX, yy = r % HY, zz = r / HY;
        int X = x0 - P + xx, Y = y0 - P + yy, Z = z0 - P + zz;
        T v = T(0);
        if (X >= 0 && X < Nx && Y >= 0 && Y < Ny && Z >= 0 && Z < Nz) v = f[Z * sxy + (long long)Y * pitch + X];
        s_in[i] = v;
      }
      cur_field = tm.field;
    }
    {
      const T* bx = prm.ax[0].band[tm.op[0]];
      const T* by = prm.ax[1].band[tm.op[1]];
      const T* bz = prm.ax[2].band[tm.op[2]];
      for (int i = tid; i < (TX + TY + TZ) * W; i += NT) {
        int row = i / W, q = i % W;
        if (row < TX) {
          int g = x0 + row;
          s_bx[row][q] = g < Nx ? bx[g * W + q] : T(0);
        } else if (row < TX + TY) {
          int g = y0 + row - TX;
          s_by[row - TX][q] = g < Ny ? by[g * W + q] : T(0);
        } else {
          int g = z0 + row - TX - TY;
          s_bz[row - TX - TY][q] = g < Nz ? bz[g * W + q] : T(0);
        }
      }
    }
    __syncthreads();
    // z pass: s_z[zz][yy][xx] = sum_q Z[z0+zz][q] s_in[zz+q][yy][xx]
    for (int i = tid; i < TZ * HY * HX; i += NT) {
      int rem = i % (HY * HX), zz = i / (HY * HX);
      T s = T(0);
#pragma unroll
      for (int q = 0; q < W; ++q) s += s_bz[zz][q] * s_in[(zz + q) * HY * HX + rem];
      s_z[i] = s;
    }
    __syncthreads();
    // y pass: s_y[zz][yy][xx] = sum_q Y[y0+yy][q] s_z[zz][yy+q][xx]
    for (int i = tid; i < TZ * TY * HX; i += NT) {
      int xx = i % HX, r = i / HX, yy = r % TY, zz = r / TY;
      T s = T(0);
#pragma unroll
      for (int q = 0; q < W; ++q) s += s_by[yy][q] * s_z[(zz * HY + yy + q) * HX + xx];
      s_y[i] = s;
    }
    __syncthreads();
    // x pass and accumulation into this thread's outputs
    const T sg = T(tm.sign);
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < W; ++q) s += s_bx[tx][q] * s_y[(zz * TY + ty) * HX + tx + q];
      T w = sg;
      switch (tm.coef) {
        case CF_A: w *= cf[1][zz]; break;
        case CF_B: w *= cf[2][zz]; break;
        case CF_C: w *= cf[3][zz]; break;
        case CF_D: w *= cf[4][zz]; break;
        default: break;
      }
      if (tm.out == 0) acc[0][zz] += w * s;
      else if (tm.out == 1) acc[1][zz] += w * s;
      else acc[2][zz] += w * s;
    }
  }

  // point source: -b amp g(t_mid) B_r(x0) B_s(y0) B_t(z0) on its component;
  // g is evaluated only by tiles that hold the source's (p+1)^3 support
  double g = 0.0;
  if (prm.src_comp >= 0 && src_in_tile(prm.src_i0, P, x0, y0, z0, TX, TY, TZ)) {
    double tm = *prm.clock_t0 + ((double)*prm.clock_step + prm.t_frac) * prm.tau;
    double u = tm - prm.src_t0;
    g = prm.src_amp * sin(2.0 * 3.14159265358979323846 * prm.src_f0 * u) * exp(-(u / prm.src_s) * (u / prm.src_s));
  }
  if (col_in) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int zz = 0; zz < TZ; ++zz) {
        int gz = z0 + zz;
        if (gz >= Nz) continue;
        T v = acc[c][zz];
        if (c == prm.src_comp) {
          int ix = gx - prm.src_i0[0], iy = gy - prm.src_i0[1], iz = gz - prm.src_i0[2];
          if (ix >= 0 && ix <= P && iy >= 0 && iy <= P && iz >= 0 && iz <= P)
            v -= cf[2][zz] * T(g) * prm.src_w[0][ix] * prm.src_w[1][iy] * prm.src_w[2][iz];
        }
        prm.out[c][gz * sxy + (long long)gy * pitch + gx] = v;
      }
    }
  }
  if (prm.advance_clock && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0)
    *prm.clock_step += 1;
}

// ---------------------------- right-hand side, material inside the integrals
// The "quad" reading of section "Incorporating non-regular material data": every
// right-hand-side term is sum_e kappa_e int_e (D_test B_rst)(D_trial u), kappa_e
// in {1, a_e, b_e, c_e, d_e} formed from the element's eps, mu, sigma (the same
// formulas as the row coefficients).  With kappa constant on each element, the
// integral over element e factorises into the element blocks of the 1D
// matrices: (X_e (x) Y_e (x) Z_e) applied to the element's (p+1)^3
// coefficients.  One CTA takes 8^3 elements (one thread each) and holds the
// coefficient tiles of all input fields.  Per output component and output
// plane c' of the element, each thread sums its element's contributions of the
// component's terms (sum factorisation inside the element, scaled by sign
// kappa_e) into (p+1)^2 registers and stores them; then every point of the
// tile gathers the contributions of the elements whose plane c' covers it
// (summed in the working precision) and adds them to an FP64 output tile (no
// atomics; the planes' partial sums meet in FP64).  The tile is finally added
// into the zeroed output arrays (neighbouring tiles share their border
// coefficients).  The source row uses b of the element that holds the dipole.
template <typename T, int P>
struct QuadTile {
  static constexpr int TE = 8, Q = P + 1, HT = TE + P, HT3 = HT * HT * HT, NE = TE * TE * TE;
  // FP64 output tiles, then (T) the element contributions of one plane, the
  // coefficient tiles of up to 9 fields and the element blocks
  static constexpr size_t OUT_B = sizeof(double) * 3 * HT3;
  static size_t bytes(int nfields) {
    return OUT_B + sizeof(T) * ((size_t)Q * Q * NE + (size_t)nfields * HT3 + (size_t)3 * TE * 4 * Q * Q);
  }
};

template <typename T, int P>
__global__ void __launch_bounds__(512) rhs_quad_kernel(const QuadParams<T> prm, int nfields) {
  using S = QuadTile<T, P>;
  constexpr int TE = S::TE, Q = S::Q, HT = S::HT, HT3 = S::HT3, NE = S::NE;
  extern __shared__ __align__(16) unsigned char quad_smem[];
  double* s_out = reinterpret_cast<double*>(quad_smem);           // [3][HT3]
  T* s_con = reinterpret_cast<T*>(quad_smem + S::OUT_B);          // [Q][Q][NE] contributions of one plane
  T* s_u = s_con + Q * Q * NE;                                     // [nfields][HT3]
  T* s_loc = s_u + nfields * HT3;                                  // [axis][element][op][test][trial]
  const int tid = threadIdx.x;
  const int lx = tid % TE, ly = (tid / TE) % TE, lz = tid / (TE * TE);
  const int e0[3] = {(int)blockIdx.x * TE, (int)blockIdx.y * TE, (int)blockIdx.z * TE};
  const int ex = e0[0] + lx, ey = e0[1] + ly, ez = e0[2] + lz;
  const bool ein = ex < prm.n[0] && ey < prm.n[1] && ez < prm.n[2];
  const int Nx = prm.Nx, Ny = prm.Ny, Nz = prm.Nz, pitch = prm.pitch;
  const long long sxy = (long long)pitch * Ny;
  for (int i = tid; i < 3 * HT3; i += NE) s_out[i] = 0.0;
  for (int i = tid; i < 3 * TE * 4 * Q * Q; i += NE) {
    const int rc = i % (Q * Q), op = (i / (Q * Q)) % 4, le = (i / (4 * Q * Q)) % TE, ax = i / (4 * Q * Q * TE);
    const int e = e0[ax] + le;
    s_loc[i] = e < prm.n[ax] ? prm.loc[ax][((long long)e * 4 + op) * Q * Q + rc] : T(0);
  }
  for (int f = 0; f < nfields; ++f) {  // coefficient tiles (8 + p)^3, zero outside the grid
    const T* __restrict__ src = prm.fields[f];
    for (int i = tid; i < HT3; i += NE) {
      const int X = e0[0] + i % HT, Y = e0[1] + (i / HT) % HT, Z = e0[2] + i / (HT * HT);
      s_u[f * HT3 + i] = (X < Nx && Y < Ny && Z < Nz) ? src[Z * sxy + (long long)Y * pitch + X] : T(0);
    }
  }
  auto loc = [&](int ax, int le, int op) { return s_loc + ((ax * TE + le) * 4 + op) * Q * Q; };
  // this element's coefficients (FP64 from the per-element material, as the row coefficients)
  double kap[5] = {1.0, 0.0, 0.0, 0.0, 0.0};  // indexed by Coef: 1, a, b, c, d
  if (ein) {
    const long long e = ((long long)ez * prm.n[1] + ey) * prm.n[0] + ex;
    const double ep = prm.eps[e], mu = prm.mu[e], sg = prm.sigma[e], tau = prm.tau;
    const double al = sg * tau / (4.0 * ep);
    kap[CF_A] = (1.0 - al) / (1.0 + al);
    kap[CF_B] = tau / (2.0 * ep * (1.0 + al));
    kap[CF_C] = tau * tau / (4.0 * ep * mu * (1.0 + al));
    kap[CF_D] = tau / (2.0 * mu);
  }
  T kapT[5];  // in the working precision, for the element products
#pragma unroll
  for (int k = 0; k < 5; ++k) kapT[k] = T(kap[k]);
  const bool src_here = prm.src_comp >= 0 && ein && ex == prm.src_e[0] && ey == prm.src_e[1] && ez == prm.src_e[2];
  double bg = 0.0;
  if (src_here) {
    const double tmid = *prm.clock_t0 + ((double)*prm.clock_step + prm.t_frac) * prm.tau;
    const double uu = tmid - prm.src_t0;
    bg = kap[CF_B] * prm.src_amp * sin(2.0 * 3.14159265358979323846 * prm.src_f0 * uu) *
         exp(-(uu / prm.src_s) * (uu / prm.src_s));
  }
  const int eoff = (lz * HT + ly) * HT + lx;  // this element's first coefficient in a tile
  __syncthreads();
  for (int comp = 0; comp < 3; ++comp) {
    for (int c2 = 0; c2 < Q; ++c2) {
      T acc[Q][Q];
#pragma unroll
      for (int b = 0; b < Q; ++b)
#pragma unroll
        for (int a = 0; a < Q; ++a) acc[b][a] = T(0);
      if (ein) {
        for (int t = 0; t < prm.nterms; ++t) {
          const Term tm = prm.terms[t];
          if (tm.out != comp) continue;
          const T* ub = s_u + tm.field * HT3 + eoff;
          const T* Zm = loc(2, lz, tm.op[2]) + c2 * Q;
          const T* Ym = loc(1, ly, tm.op[1]);
          const T* Xm = loc(0, lx, tm.op[0]);
          const T w = T(tm.sign) * kapT[tm.coef];
          T t1[Q][Q];
#pragma unroll
          for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int a = 0; a < Q; ++a) {
              T sm = T(0);
#pragma unroll
              for (int k = 0; k < Q; ++k) sm += Zm[k] * ub[(k * HT + b) * HT + a];
              t1[b][a] = sm;
            }
#pragma unroll
          for (int b2 = 0; b2 < Q; ++b2) {
            T t2[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
              T sm = T(0);
#pragma unroll
              for (int k = 0; k < Q; ++k) sm += Ym[b2 * Q + k] * t1[k][a];
              t2[a] = sm;
            }
#pragma unroll
            for (int a2 = 0; a2 < Q; ++a2) {
              T sm = T(0);
#pragma unroll
              for (int k = 0; k < Q; ++k) sm += Xm[a2 * Q + k] * t2[k];
              acc[b2][a2] += w * sm;
            }
          }
        }
        if (src_here && comp == prm.src_comp) {
#pragma unroll
          for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int a = 0; a < Q; ++a)
              acc[b][a] -= T(bg * (double)prm.src_w[0][a] * (double)prm.src_w[1][b] * (double)prm.src_w[2][c2]);
        }
      }
#pragma unroll
      for (int b = 0; b < Q; ++b)
#pragma unroll
        for (int a = 0; a < Q; ++a) s_con[(b * Q + a) * NE + tid] = ein ? acc[b][a] : T(0);
      __syncthreads();
      // every tile point (Z, Y, X) of plane offset c2 gathers from the elements (Z - c2, Y - b, X - a)
      for (int i = tid; i < HT3; i += NE) {
        const int X = i % HT, Y = (i / HT) % HT, Z = i / (HT * HT);
        const int zl = Z - c2;
        if (zl < 0 || zl >= TE) continue;
        T sm = T(0);  // the (p+1)^2 contributions of this plane in T, the planes in FP64
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          const int yl = Y - b;
          if (yl < 0 || yl >= TE) continue;
#pragma unroll
          for (int a = 0; a < Q; ++a) {
            const int xl = X - a;
            if (xl < 0 || xl >= TE) continue;
            sm += s_con[(b * Q + a) * NE + (zl * TE + yl) * TE + xl];
          }
        }
        s_out[comp * HT3 + i] += (double)sm;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < HT3; i += NE) {
    const int X = e0[0] + i % HT, Y = e0[1] + (i / HT) % HT, Z = e0[2] + i / (HT * HT);
    if (X >= Nx || Y >= Ny || Z >= Nz) continue;
    const long long g = Z * sxy + (long long)Y * pitch + X;
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(prm.out[c] + g, T(s_out[c * HT3 + i]));  // result unused: a reduction in L2
  }
}

// ------------------------------------- mixed-mode E right-hand side (BF16 MMA)
// The contraction of eq. dupa1ab (and its half-step-2 analogue) with BF16
// operands on the tensor cores: per 32 x 8 x 8 output tile and Kronecker term,
// the first pass (along x) is a GEMM
//     X[(z, y)][xo] = sum_k T[(z, y)][k] * Wx^T[k][xo]
// of the haloed field tile T (rows: the (z, y) pairs of the haloed tile, k: the
// haloed x index, both BF16: the field rounded to BF16) with the banded 1D
// operator of the term's x factor (BF16), accumulated in FP32 by
// mma.sync.m16n8k16 (M = 16 tile rows, N = 8 outputs, K = 16 haloed x values;
// K is padded from 32 + 2p to 48 with zeros).  A operands come from shared
// memory by ldmatrix, B operands are built in registers from the band table.
// The y and z passes and the row scaling by a, b, c then run in FP32 on the
// CUDA cores from the FP32 partial sums.  The refinement that follows (float-
// float or FP64 residual) removes the BF16 error of this contraction.
template <int P>
struct MmaTile {
  static constexpr int TX = 32, TY = 8, TZ = 8;
  static constexpr int HX = TX + 2 * P, HY = TY + 2 * P, HZ = TZ + 2 * P;
  static constexpr int ROWS = HZ * HY;               // (z, y) rows of the haloed tile
  static constexpr int MT = (ROWS + 15) / 16;        // m tiles of 16 rows
  static constexpr int KS = 3;                       // k steps of 16 (K padded to 48 >= HX)
  static constexpr int TS = 56;                      // BF16 tile row stride (112 B: conflict-free ldmatrix)
  static constexpr int XS = 36;                      // FP32 row stride of the x-pass result
  static constexpr size_t TILE_B = sizeof(__nv_bfloat16) * (size_t)MT * 16 * TS;
  static constexpr size_t X_B = sizeof(float) * (size_t)ROWS * XS;
  static constexpr size_t Y_B = sizeof(float) * (size_t)HZ * TY * TX;
  // B fragments of the three x operators M, A, B: [op][n tile][k step][half][lane]
  static constexpr size_t BF_B = sizeof(unsigned) * 3 * 4 * KS * 2 * 32;
  static constexpr size_t BYTES = TILE_B + X_B + Y_B + BF_B;
  static_assert(HX <= 16 * KS, "x halo exceeds the padded K");
};

__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (lower address)
  return *reinterpret_cast<const unsigned*>(&v);
}

template <int P>
__global__ void __launch_bounds__(256) rhs_e_mma_kernel(const RhsParams<float> prm) {
  using S = MmaTile<P>;
  constexpr int TX = S::TX, TY = S::TY, TZ = S::TZ, HX = S::HX, HY = S::HY, HZ = S::HZ;
  constexpr int W = 2 * P + 1;
  constexpr int NT = TX * TY;
  extern __shared__ __align__(16) unsigned char mma_smem[];
  __nv_bfloat16* s_tile = reinterpret_cast<__nv_bfloat16*>(mma_smem);
  float* s_x = reinterpret_cast<float*>(mma_smem + S::TILE_B);
  float* s_y = reinterpret_cast<float*>(mma_smem + S::TILE_B + S::X_B);
  unsigned* s_bf = reinterpret_cast<unsigned*>(mma_smem + S::TILE_B + S::X_B + S::Y_B);
  __shared__ float s_by[TY][W], s_bz[TZ][W];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int Nx = prm.Nx, Ny = prm.Ny, Nz = prm.Nz, pitch = prm.pitch;
  const long long sxy = (long long)pitch * Ny;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool col_in = gx < Nx && gy < Ny;

  float cf[4][TZ];  // 1, a, b, c
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz) {
    const int gz = z0 + zz;
    const bool in = col_in && gz < Nz;
    const long long g = gz * sxy + (long long)gy * pitch + gx;
    cf[0][zz] = 1.f;
#pragma unroll
    for (int k = 1; k < 4; ++k) cf[k][zz] = in && prm.coef[k] ? prm.coef[k][g] : 0.f;
  }
  float acc[3][TZ];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) acc[c][zz] = 0.f;

  // zero the padding of the BF16 tile once: columns HX .. TS-1 and rows ROWS .. 16 MT - 1
  for (int i = tid; i < S::MT * 16 * S::TS; i += NT) {
    const int r = i / S::TS, k = i % S::TS;
    if (k >= HX || r >= S::ROWS) s_tile[i] = __float2bfloat16(0.f);
  }
  // B fragments of this tile's x operators (the same for every term that uses
  // the operator): B[k][n] = Wx[x0+n][k - n] (band index), BF16; lane l holds
  // k = 2(l % 4) + {0, 1} (+ 8 for the second register), n = l / 4 (+ 8 nt)
  for (int i = tid; i < 3 * 4 * S::KS * 2 * 32; i += NT) {
    const int ln = i % 32, h = (i / 32) % 2, ks = (i / 64) % S::KS, nt = (i / (64 * S::KS)) % 4;
    const int oi = i / (64 * S::KS * 4);
    const float* bx = prm.ax[0].band[oi == 0 ? OP_M : (oi == 1 ? OP_A : OP_B)];
    const int n = nt * 8 + (ln >> 2);
    float v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int q = ks * 16 + h * 8 + 2 * (ln & 3) + e - n;
      v[e] = (x0 + n < Nx && q >= 0 && q < W) ? bx[(x0 + n) * W + q] : 0.f;
    }
    s_bf[i] = pack_bf16x2(v[0], v[1]);
  }

  int cur_field = -1;
  for (int t = 0; t < prm.nterms; ++t) {
    const Term tm = prm.terms[t];
    __syncthreads();  // previous term done with s_tile / s_x / s_y / band rows
    if (tm.field != cur_field) {  // the haloed field tile, rounded to BF16
      const float* __restrict__ f = prm.fields[tm.field];
      for (int i = tid; i < S::ROWS * HX; i += NT) {
        const int xx = i % HX, r = i / HX, yy = r % HY, zz = r / HY;
        const int X = x0 - P + xx, Y = y0 - P + yy, Z = z0 - P + zz;
        float v = 0.f;
        if (X >= 0 && X < Nx && Y >= 0 && Y < Ny && Z >= 0 && Z < Nz) v = f[Z * sxy + (long long)Y * pitch + X];
        s_tile[r * S::TS + xx] = __float2bfloat16(v);
      }
      cur_field = tm.field;
    }
    {
      const float* by = prm.ax[1].band[tm.op[1]];
      const float* bz = prm.ax[2].band[tm.op[2]];
      for (int i = tid; i < (TY + TZ) * W; i += NT) {
        const int row = i / W, q = i % W;
        if (row < TY) {
          const int g = y0 + row;
          s_by[row][q] = g < Ny ? by[g * W + q] : 0.f;
        } else {
          const int g = z0 + row - TY;
          s_bz[row - TY][q] = g < Nz ? bz[g * W + q] : 0.f;
        }
      }
    }
    const unsigned* bf = s_bf + (tm.op[0] == OP_M ? 0 : (tm.op[0] == OP_A ? 1 : 2)) * (4 * S::KS * 2 * 32) + lane;
    __syncthreads();
    // x pass on the tensor cores: warp w takes m tiles w, w + 8, ...
    for (int mt = warp; mt < S::MT; mt += NT / 32) {
      unsigned afr[S::KS][4];
      {
        const int mi = lane >> 3, r8 = lane & 7;
        const int row = mt * 16 + r8 + (mi & 1) * 8;
#pragma unroll
        for (int ks = 0; ks < S::KS; ++ks) {
          const unsigned addr = (unsigned)__cvta_generic_to_shared(s_tile + row * S::TS + ks * 16 + (mi >> 1) * 8);
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                       : "=r"(afr[ks][0]), "=r"(afr[ks][1]), "=r"(afr[ks][2]), "=r"(afr[ks][3])
                       : "r"(addr));
        }
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < S::KS; ++ks)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
              "{%0, %1, %2, %3};\n"
              : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
              : "r"(afr[ks][0]), "r"(afr[ks][1]), "r"(afr[ks][2]), "r"(afr[ks][3]),
                "r"(bf[((nt * S::KS + ks) * 2 + 0) * 32]), "r"(bf[((nt * S::KS + ks) * 2 + 1) * 32]));
        const int g4 = lane >> 2, t4 = lane & 3;
        const int r0 = mt * 16 + g4, c0 = nt * 8 + 2 * t4;
        if (r0 < S::ROWS) {
          s_x[r0 * S::XS + c0] = d[0];
          s_x[r0 * S::XS + c0 + 1] = d[1];
        }
        if (r0 + 8 < S::ROWS) {
          s_x[(r0 + 8) * S::XS + c0] = d[2];
          s_x[(r0 + 8) * S::XS + c0 + 1] = d[3];
        }
      }
    }
    __syncthreads();
    // y pass (FP32): s_y[zh][yo][xo] = sum_q Wy[yo][q] X[(zh, yo + q)][xo]
    for (int i = tid; i < HZ * TY * TX; i += NT) {
      const int xo = i % TX, r = i / TX, yo = r % TY, zh = r / TY;
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < W; ++q) v += s_by[yo][q] * s_x[(zh * HY + yo + q) * S::XS + xo];
      s_y[i] = v;
    }
    __syncthreads();
    // z pass (FP32) and accumulation into this thread's outputs
    const float sg = tm.sign;
    const int ck = tm.coef == CF_A ? 1 : tm.coef == CF_B ? 2 : tm.coef == CF_C ? 3 : 0;
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < W; ++q) v += s_bz[zz][q] * s_y[((zz + q) * TY + ty) * TX + tx];
      const float w = sg * cf[ck][zz] * v;
      if (tm.out == 0) acc[0][zz] += w;
      else if (tm.out == 1) acc[1][zz] += w;
      else acc[2][zz] += w;
    }
  }

  // point source: -b amp g(t_mid) B_r(x0) B_s(y0) B_t(z0) on its component
  double g = 0.0;
  if (prm.src_comp >= 0 && src_in_tile(prm.src_i0, P, x0, y0, z0, TX, TY, TZ)) {
    const double tmid = *prm.clock_t0 + ((double)*prm.clock_step + prm.t_frac) * prm.tau;
    const double u = tmid - prm.src_t0;
    g = prm.src_amp * sin(2.0 * 3.14159265358979323846 * prm.src_f0 * u) * exp(-(u / prm.src_s) * (u / prm.src_s));
  }
  if (!col_in) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      const int gz = z0 + zz;
      if (gz >= Nz) continue;
      float v = acc[c][zz];
      if (c == prm.src_comp) {
        const int ix = gx - prm.src_i0[0], iy = gy - prm.src_i0[1], iz = gz - prm.src_i0[2];
        if (ix >= 0 && ix <= P && iy >= 0 && iy <= P && iz >= 0 && iz <= P)
          v -= cf[2][zz] * (float)g * prm.src_w[0][ix] * prm.src_w[1][iy] * prm.src_w[2][iz];
      }
      prm.out[c][gz * sxy + (long long)gy * pitch + gx] = v;
    }
  }
}

// ------------------------------------------------ mixed-mode FP64 residual
// r = RHS - T E* of the E system, in FP64 arithmetic from FP32 arrays:
// fields 0..5 are the inputs of the E right-hand side (E, H of the old level),
// 6..8 the FP32 solution E* of T E = RHS(BF16 tiles); the terms are the 12 of
// the right-hand side and, per component, -M(x)M(x)M E*_k and -c S_s(x)M(x)M
// E*_k (S along the stiffness axis s of component k).  Same tiling as
// rhs_kernel; band tables in FP64.
struct ResidParams {
  const float* fields[9];
  const float* coef[5];  // [CF_A], [CF_B], [CF_C]
  float* out[3];
  const double* band[3][4];  // [axis][op]
  Term terms[kMaxResidTerms];
  int nterms;
  int Nx, Ny, Nz, pitch;
  int src_comp;
  int src_i0[3];
  double src_w[3][kMaxP + 1];
  double src_amp, src_f0, src_t0, src_s;
  double tau, t_frac;
  const double* clock_t0;
  const long long* clock_step;
};

template <int P>
__global__ void __launch_bounds__(256) resid_kernel(const ResidParams prm) {
  constexpr int TX = 32, TY = 8, TZ = 8;
  constexpr int W = 2 * P + 1;
  constexpr int HX = TX + 2 * P, HY = TY + 2 * P, HZ = TZ + 2 * P;
  constexpr int NT = TX * TY;
  extern __shared__ __align__(16) unsigned char resid_smem[];
  double* s_in = reinterpret_cast<double*>(resid_smem);
  double* s_z = s_in + HZ * HY * HX;
  double* s_y = s_z + TZ * HY * HX;
  __shared__ double s_bx[TX][W], s_by[TY][W], s_bz[TZ][W];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int Nx = prm.Nx, Ny = prm.Ny, Nz = prm.Nz, pitch = prm.pitch;
  const long long sxy = (long long)pitch * Ny;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool col_in = gx < Nx && gy < Ny;
  double cf[4][TZ];  // 1, a, b, c
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz) {
    const int gz = z0 + zz;
    const bool in = col_in && gz < Nz;
    const long long g = gz * sxy + (long long)gy * pitch + gx;
    cf[0][zz] = 1.0;
#pragma unroll
    for (int k = 1; k < 4; ++k) cf[k][zz] = in ? (double)prm.coef[k][g] : 0.0;
  }
  double acc[3][TZ];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) acc[c][zz] = 0.0;
  int cur_field = -1;
  for (int t = 0; t < prm.nterms; ++t) {
    const Term tm = prm.terms[t];
    __syncthreads();
    if (tm.field != cur_field) {
      const float* __restrict__ f = prm.fields[tm.field];
      for (int i = tid; i < HZ * HY * HX; i += NT) {
        const int xx = i % HX, r = i / HX, yy = r % HY, zz = r / HY;
        const int X = x0 - P + xx, Y = y0 - P + yy, Z = z0 - P + zz;
        double v = 0.0;
        if (X >= 0 && X < Nx && Y >= 0 && Y < Ny && Z >= 0 && Z < Nz) v = f[Z * sxy + (long long)Y * pitch + X];
        s_in[i] = v;
      }
      cur_field = tm.field;
    }
    {
      const double* bx = prm.band[0][tm.op[0]];
      const double* by = prm.band[1][tm.op[1]];
      const double* bz = prm.band[2][tm.op[2]];
      for (int i = tid; i < (TX + TY + TZ) * W; i += NT) {
        const int row = i / W, q = i % W;
        if (row < TX) {
          const int g = x0 + row;
          s_bx[row][q] = g < Nx ? bx[g * W + q] : 0.0;
        } else if (row < TX + TY) {
          const int g = y0 + row - TX;
          s_by[row - TX][q] = g < Ny ? by[g * W + q] : 0.0;
        } else {
          const int g = z0 + row - TX - TY;
          s_bz[row - TX - TY][q] = g < Nz ? bz[g * W + q] : 0.0;
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < TZ * HY * HX; i += NT) {
      const int rem = i % (HY * HX), zz = i / (HY * HX);
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < W; ++q) v += s_bz[zz][q] * s_in[(zz + q) * HY * HX + rem];
      s_z[i] = v;
    }
    __syncthreads();
    for (int i = tid; i < TZ * TY * HX; i += NT) {
      const int xx = i % HX, r = i / HX, yy = r % TY, zz = r / TY;
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < W; ++q) v += s_by[yy][q] * s_z[(zz * HY + yy + q) * HX + xx];
      s_y[i] = v;
    }
    __syncthreads();
    const int ck = tm.coef == CF_A ? 1 : tm.coef == CF_B ? 2 : tm.coef == CF_C ? 3 : 0;
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < W; ++q) v += s_bx[tx][q] * s_y[(zz * TY + ty) * HX + tx + q];
      const double w = (double)tm.sign * cf[ck][zz] * v;
      if (tm.out == 0) acc[0][zz] += w;
      else if (tm.out == 1) acc[1][zz] += w;
      else acc[2][zz] += w;
    }
  }
  double g = 0.0;
  if (prm.src_comp >= 0 && src_in_tile(prm.src_i0, P, x0, y0, z0, TX, TY, TZ)) {
    const double tmid = *prm.clock_t0 + ((double)*prm.clock_step + prm.t_frac) * prm.tau;
    const double u = tmid - prm.src_t0;
    g = prm.src_amp * sin(2.0 * 3.14159265358979323846 * prm.src_f0 * u) * exp(-(u / prm.src_s) * (u / prm.src_s));
  }
  if (!col_in) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      const int gz = z0 + zz;
      if (gz >= Nz) continue;
      double v = acc[c][zz];
      if (c == prm.src_comp) {
        const int ix = gx - prm.src_i0[0], iy = gy - prm.src_i0[1], iz = gz - prm.src_i0[2];
        if (ix >= 0 && ix <= P && iy >= 0 && iy <= P && iz >= 0 && iz <= P)
          v -= cf[2][zz] * g * prm.src_w[0][ix] * prm.src_w[1][iy] * prm.src_w[2][iz];
      }
      prm.out[c][gz * sxy + (long long)gy * pitch + gx] = (float)v;
    }
  }
}

// ------------------------------------- mixed-mode float-float residual
// The same residual r = RHS - T E* as resid_kernel, evaluated in compensated
// double-float arithmetic on the FP32 pipe instead of the FP64 pipe (GB300 runs
// FP64 at 1/64 of the FP32 rate).  A value is an unevaluated sum hi + lo of two
// floats (about 48 significant bits).  The error-free transformations are the
// published ones: TwoSum (Knuth, TAOCP vol. 2: s = a + b and its exact
// rounding error, six additions) and TwoProduct by fused multiply-add (the
// product's rounding error is fma(a, b, -a*b); Dekker's product, 1971, without
// splitting); sums of double-float values renormalise with Fast-TwoSum.  The
// roundings are explicit (__fadd_rn / __fmul_rn), so the compiler cannot fuse
// them into FMAs that would break the transformations.  The fields and the
// row coefficients are FP32 (exact as double-float), the band tables are the
// FP64 tables split into hi + lo on the host.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// sum of two double-float values: TwoSum of the high parts, the low parts added
// to its error, renormalised (error about 2^-44 of |a| + |b|)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
// a * b for a double-float a and a float b
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return ff_fast_two_sum(p, e);
}

struct ResidFFParams {
  const float* fields[9];
  const float* coef[5];  // [CF_A], [CF_B], [CF_C]
  float* out[3];
  const float2* band[3][4];  // [axis][op]: (hi, lo) of the FP64 band tables
  Term terms[kMaxResidTerms];
  int nterms;
  int Nx, Ny, Nz, pitch;
  int src_comp;
  int src_i0[3];
  double src_w[3][kMaxP + 1];
  double src_amp, src_f0, src_t0, src_s;
  double tau, t_frac;
  const double* clock_t0;
  const long long* clock_step;
};

template <int P>
__global__ void __launch_bounds__(256) resid_ff_kernel(const ResidFFParams prm) {
  constexpr int TX = 32, TY = 8, TZ = 8;
  constexpr int W = 2 * P + 1;
  constexpr int HX = TX + 2 * P, HY = TY + 2 * P, HZ = TZ + 2 * P;
  constexpr int NT = TX * TY;
  extern __shared__ __align__(16) unsigned char resid_ff_smem[];
  float* s_in = reinterpret_cast<float*>(resid_ff_smem);              // FP32 inputs (exact)
  ff* s_z = reinterpret_cast<ff*>(s_in + ((HZ * HY * HX + 1) & ~1));  // z pass, double-float
  ff* s_y = s_z + TZ * HY * HX;                                       // y pass
  __shared__ ff s_bx[TX][W], s_by[TY][W], s_bz[TZ][W];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int Nx = prm.Nx, Ny = prm.Ny, Nz = prm.Nz, pitch = prm.pitch;
  const long long sxy = (long long)pitch * Ny;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool col_in = gx < Nx && gy < Ny;
  float cf[4][TZ];  // 1, a, b, c (FP32 arrays: exact)
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz) {
    const int gz = z0 + zz;
    const bool in = col_in && gz < Nz;
    const long long g = gz * sxy + (long long)gy * pitch + gx;
    cf[0][zz] = 1.f;
#pragma unroll
    for (int k = 1; k < 4; ++k) cf[k][zz] = in ? prm.coef[k][g] : 0.f;
  }
  ff acc[3][TZ];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) acc[c][zz] = ff{0.f, 0.f};
  int cur_field = -1;
  for (int t = 0; t < prm.nterms; ++t) {
    const Term tm = prm.terms[t];
    __syncthreads();
    if (tm.field != cur_field) {
      const float* __restrict__ f = prm.fields[tm.field];
      for (int i = tid; i < HZ * HY * HX; i += NT) {
        const int xx = i % HX, r = i / HX, yy = r % HY, zz = r / HY;
        const int X = x0 - P + xx, Y = y0 - P + yy, Z = z0 - P + zz;
        float v = 0.f;
        if (X >= 0 && X < Nx && Y >= 0 && Y < Ny && Z >= 0 && Z < Nz) v = f[Z * sxy + (long long)Y * pitch + X];
        s_in[i] = v;
      }
      cur_field = tm.field;
    }
    {
      const float2* bx = prm.band[0][tm.op[0]];
      const float2* by = prm.band[1][tm.op[1]];
      const float2* bz = prm.band[2][tm.op[2]];
      for (int i = tid; i < (TX + TY + TZ) * W; i += NT) {
        const int row = i / W, q = i % W;
        float2 v = make_float2(0.f, 0.f);
        if (row < TX) {
          const int g = x0 + row;
          if (g < Nx) v = bx[g * W + q];
          s_bx[row][q] = ff{v.x, v.y};
        } else if (row < TX + TY) {
          const int g = y0 + row - TX;
          if (g < Ny) v = by[g * W + q];
          s_by[row - TX][q] = ff{v.x, v.y};
        } else {
          const int g = z0 + row - TX - TY;
          if (g < Nz) v = bz[g * W + q];
          s_bz[row - TX - TY][q] = ff{v.x, v.y};
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < TZ * HY * HX; i += NT) {
      const int rem = i % (HY * HX), zz = i / (HY * HX);
      ff v{0.f, 0.f};
#pragma unroll
      for (int q = 0; q < W; ++q) v = ff_add(v, ff_mul_f(s_bz[zz][q], s_in[(zz + q) * HY * HX + rem]));
      s_z[i] = v;
    }
    __syncthreads();
    for (int i = tid; i < TZ * TY * HX; i += NT) {
      const int xx = i % HX, r = i / HX, yy = r % TY, zz = r / TY;
      ff v{0.f, 0.f};
#pragma unroll
      for (int q = 0; q < W; ++q) v = ff_add(v, ff_mul(s_by[yy][q], s_z[(zz * HY + yy + q) * HX + xx]));
      s_y[i] = v;
    }
    __syncthreads();
    const int ck = tm.coef == CF_A ? 1 : tm.coef == CF_B ? 2 : tm.coef == CF_C ? 3 : 0;
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      ff v{0.f, 0.f};
#pragma unroll
      for (int q = 0; q < W; ++q) v = ff_add(v, ff_mul(s_bx[tx][q], s_y[(zz * TY + ty) * HX + tx + q]));
      ff w = ff_mul_f(v, tm.sign * cf[ck][zz]);  // sign is +-1: exact
      if (tm.out == 0) acc[0][zz] = ff_add(acc[0][zz], w);
      else if (tm.out == 1) acc[1][zz] = ff_add(acc[1][zz], w);
      else acc[2][zz] = ff_add(acc[2][zz], w);
    }
  }
  double g = 0.0;
  if (prm.src_comp >= 0 && src_in_tile(prm.src_i0, P, x0, y0, z0, TX, TY, TZ)) {
    const double tmid = *prm.clock_t0 + ((double)*prm.clock_step + prm.t_frac) * prm.tau;
    const double u = tmid - prm.src_t0;
    g = prm.src_amp * sin(2.0 * 3.14159265358979323846 * prm.src_f0 * u) * exp(-(u / prm.src_s) * (u / prm.src_s));
  }
  if (!col_in) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int zz = 0; zz < TZ; ++zz) {
      const int gz = z0 + zz;
      if (gz >= Nz) continue;
      ff v = acc[c][zz];
      if (c == prm.src_comp) {
        const int ix = gx - prm.src_i0[0], iy = gy - prm.src_i0[1], iz = gz - prm.src_i0[2];
        if (ix >= 0 && ix <= P && iy >= 0 && iy <= P && iz >= 0 && iz <= P) {
          // the source row (one point per tile) in FP64, split into hi + lo
          const double sv = (double)cf[2][zz] * g * prm.src_w[0][ix] * prm.src_w[1][iy] * prm.src_w[2][iz];
          const float sh = (float)sv;
          v = ff_add(v, ff{-sh, -(float)(sv - (double)sh)});
        }
      }
      prm.out[c][gz * sxy + (long long)gy * pitch + gx] = __fadd_rn(v.hi, v.lo);
    }
  }
}

// E += delta on the N_x columns of every row (mixed-mode refinement)
__global__ void add_delta_kernel(float* e0, float* e1, float* e2, const float* d0, const float* d1,
                                 const float* d2, int Nx, int pitch, long long rows) {
  const long long n = rows * (long long)Nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long g = (i / Nx) * pitch + i % Nx;
    e0[g] += d0[g];
    e1[g] += d1[g];
    e2[g] += d2[g];
  }
}

// ----------------------------------------------------------- line solves
// Asynchronous global -> shared copy of one element (cp.async, no register
// round trip); all copies of a tile are in flight together.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// Fire-and-forget global add (red.global.add): the L2 performs the update.
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;\n" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;\n" ::"l"(p), "d"(v) : "memory");
}

// Banded solves along one axis, one thread per line (Gaussian elimination
// without pivoting restricted to the band; Appendix, eqs. split1/split2).
//   LM_MASS : dst = M^-1 src with the precomputed (full or Dirichlet) mass LU.
//   LM_STIFF: dst = (M + diag(c) S)^-1 src; the LU of each line is formed row
//             by row from c (per-test-function material) and the inverse
//             pivots of an LM_PIVOT pass (they depend only on c and tau), so
//             no reciprocal lies on the recurrence; the normalised upper factors
//             are kept in shared memory for the back substitution.
//   LM_DERIV: dst += scale * M^-1 (A src): the 1D derivative in the L2 sense,
//             added in place with red.global.add (H half steps, uniform mu).
//   LM_PIVOT: dst = 1 / pivots of the LU of M + diag(c) S (run once per dt).
// A tile of LINES lines is staged with cp.async into shared memory as
// [row][line] (x lines transposed; pitch LINES+1 for x so both the staging and
// the per-thread recurrence are bank-conflict free), solved in place, written
// back.  The 1D tables of the axis are staged into shared memory; rows whose
// factors equal the mid-line factors in T use register constants instead.
// blockIdx.y selects one of up to three independent jobs on the same axis.
template <typename T, int P, int MODE, bool XDIR>
__global__ void __launch_bounds__(64) line_kernel(const LineJobs<T> jobs, const LineParams lp, const AxisDev<T> ax) {
  constexpr int W = 2 * P + 1;
  constexpr bool FACT = MODE == LM_STIFF || MODE == LM_PIVOT;  // works on M + c S
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // static parameter offsets (a dynamic index would copy the struct to the stack)
  const LineJob<T> job = blockIdx.y == 0 ? jobs.job[0] : (blockIdx.y == 1 ? jobs.job[1] : jobs.job[2]);
  const int dch = job.dirichlet;
  const int LINES = blockDim.x, LP = XDIR ? LINES + 1 : LINES, N = lp.N;
  constexpr int TABW = FACT ? 2 * W : (MODE == LM_DERIV ? 3 * P + 1 + W : 3 * P + 1);
  T* tab = reinterpret_cast<T*>(smem_raw);
  T* sr = tab + ((N * TABW + 3) & ~3);  // [N][LP]: rhs, then y', then x (PIVOT: 1/pivot)
  T* su = sr + N * LP;                  // FACT: c; STIFF: 1/pivot, then the P upper-factor planes
  const int plane = N * LP;
  const int t = threadIdx.x;
  const int L0 = blockIdx.x * LINES;
  const int cnt = min(LINES, (int)(lp.nlines - L0));

  // ---- 1D tables: MASS/DERIV [L(P) inv U(P) (A(W))], FACT [M(W) S(W)], row-major per row
  // (asynchronous, in flight together with the tile below)
  for (int i = t; i < N; i += LINES) {
    T* row = tab + i * TABW;
    if (FACT) {
#pragma unroll
      for (int d = 0; d < W; ++d) {
        cp_async_elem(&row[d], &ax.band[OP_M][i * W + d]);
        cp_async_elem(&row[W + d], &ax.band[OP_S][i * W + d]);
      }
    } else {
      const T* Lt = dch ? ax.luL[1] : ax.luL[0];
      const T* It = dch ? ax.luInv[1] : ax.luInv[0];
      const T* Ut = dch ? ax.luU[1] : ax.luU[0];
#pragma unroll
      for (int q = 0; q < P; ++q) {
        cp_async_elem(&row[q], &Lt[i * P + q]);
        cp_async_elem(&row[P + 1 + q], &Ut[i * P + q]);
      }
      cp_async_elem(&row[P], &It[i]);
      if (MODE == LM_DERIV) {
#pragma unroll
        for (int d = 0; d < W; ++d) cp_async_elem(&row[3 * P + 1 + d], &ax.band[OP_A][i * W + d]);
      }
    }
  }

  // ---- stage the tile: src (not PIVOT), c (FACT), inverse pivots (STIFF)
  const T* in0 = MODE == LM_PIVOT ? nullptr : job.src;
  const T* in1 = FACT ? job.aux : nullptr;
  const T* in2 = MODE == LM_STIFF ? job.aux2 : nullptr;
  T* s2 = su + plane;  // STIFF: staging plane of the inverse pivots
  long long off = 0, stride = 1;  // first element and stride of this thread's line (columns)
  if (XDIR) {
    const long long b0 = (long long)L0 * lp.pitch;
    for (int line = 0; line < cnt; ++line) {
      const long long g = b0 + (long long)line * lp.pitch;
      for (int k = t; k < N; k += LINES) {
        if (MODE != LM_PIVOT) cp_async_elem(&sr[k * LP + line], in0 + g + k);
        if (FACT) cp_async_elem(&su[k * LP + line], in1 + g + k);
        if (MODE == LM_STIFF) cp_async_elem(&s2[k * LP + line], in2 + g + k);
      }
    }
  } else if (t < cnt) {
    const int L = L0 + t;
    if (lp.dir == 1) {  // line L = z * N_x + x
      off = (long long)(L / lp.Nx) * lp.pitch * lp.Ny + (L % lp.Nx);
      stride = lp.pitch;
    } else {            // line L = y * N_x + x
      off = (long long)(L / lp.Nx) * lp.pitch + (L % lp.Nx);
      stride = (long long)lp.pitch * lp.Ny;
    }
    long long g = off;
#pragma unroll 8
    for (int k = 0; k < N; ++k) {
      if (MODE != LM_PIVOT) cp_async_elem(&sr[k * LP + t], in0 + g);
      if (FACT) cp_async_elem(&su[k * LP + t], in1 + g);
      if (MODE == LM_STIFF) cp_async_elem(&s2[k * LP + t], in2 + g);
      g += stride;
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // y / z lines (one line per thread, own column): the backward sweep stores each
  // result row directly (coalesced across the warp) instead of a write-back pass
  constexpr bool FUSED = !XDIR && MODE != LM_PIVOT;
  T* gdst = job.dst + off;
  if (t < cnt) {
    const int lo = dch ? 1 : 0, hi = dch ? N - 2 : N - 1;
    T* col = sr + t;
    const long long gfac = XDIR ? (long long)(L0 + t) * lp.pitch : off;  // this line in the state layout
    const long long sfac = XDIR ? 1 : stride;
    (void)gfac;
    (void)sfac;
    if (FACT) {
      T Uq[P][P + 1], invq[P], yq[P];
#pragma unroll
      for (int m = 0; m < P; ++m) {
        invq[m] = T(0);
        yq[m] = T(0);
#pragma unroll
        for (int e = 0; e <= P; ++e) Uq[m][e] = T(0);
      }
      // one row of the Doolittle LU of M + c S (and, for STIFF, the forward step)
      auto row = [&](int k, bool inner, T ck, T rk, T ik) {
        const T* tb = tab + k * TABW;
        T a[W];
#pragma unroll
        for (int d = 0; d < W; ++d) {
          const T mv = inner ? ax.inner[OP_M][d] : tb[d];
          const T sv = inner ? ax.inner[OP_S][d] : tb[W + d];
          a[d] = mv + ck * sv;
          if (!inner) {
            const int j = k + d - P;
            if (j < lo || j > hi) a[d] = T(0);
          }
        }
        T l[P + 1];
        l[0] = T(0);
#pragma unroll
        for (int q = P; q >= 1; --q) {  // multiplier of row k - q
          T s = a[P - q];
#pragma unroll
          for (int m = q + 1; m <= P; ++m) s -= l[m] * Uq[m - 1][m - q];
          l[q] = s * invq[q - 1];
        }
        T Un[P + 1];
#pragma unroll
        for (int e = 0; e <= P; ++e) {
          T s = a[P + e];
#pragma unroll
          for (int m = 1; m <= P; ++m)
            if (e + m <= P) s -= l[m] * Uq[m - 1][e + m];
          Un[e] = s;
        }
        T inv;
        if (MODE == LM_PIVOT) {
          inv = fast_rcp(Un[0]);
          col[k * LP] = inv;
          if (job.fac[0]) {  // row factors for the streaming stiffness solve
            const long long g = gfac + k * sfac;
#pragma unroll
            for (int q = 1; q <= P; ++q) job.fac[q - 1][g] = l[q];
#pragma unroll
            for (int e = 1; e <= P; ++e) job.fac[P + e - 1][g] = Un[e] * inv;
          }
        } else {
          inv = ik;
          T y = rk;
#pragma unroll
          for (int m = 1; m <= P; ++m) y -= l[m] * yq[m - 1];
          col[k * LP] = y * inv;
#pragma unroll
          for (int e = 1; e <= P; ++e) su[(e - 1) * plane + k * LP + t] = Un[e] * inv;
#pragma unroll
          for (int m = P - 1; m >= 1; --m) yq[m] = yq[m - 1];
          yq[0] = y;
        }
#pragma unroll
        for (int m = P - 1; m >= 1; --m) {
          invq[m] = invq[m - 1];
#pragma unroll
          for (int e = 0; e <= P; ++e) Uq[m][e] = Uq[m - 1][e];
        }
        invq[0] = inv;
#pragma unroll
        for (int e = 0; e <= P; ++e) Uq[0][e] = Un[e];
      };
      // rows whose band lies inside the solved range and in the interior stencil
      const int kin0 = max(lo + P, ax.inner_lo), kin1 = min(hi - P, ax.inner_hi);
      auto row1 = [&](int k, bool inner) {
        row(k, inner, su[k * LP + t], MODE == LM_STIFF ? col[k * LP] : T(0),
            MODE == LM_STIFF ? s2[k * LP + t] : T(0));
      };
      int k = lo;
      for (; k < kin0 && k <= hi; ++k) row1(k, false);
      // interior rows in blocks of 4: all loads of a block precede its stores
      for (; k + 3 <= kin1; k += 4) {
        T cc[4], rr[4], ii[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          cc[u] = su[(k + u) * LP + t];
          rr[u] = MODE == LM_STIFF ? col[(k + u) * LP] : T(0);
          ii[u] = MODE == LM_STIFF ? s2[(k + u) * LP + t] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) row(k + u, true, cc[u], rr[u], ii[u]);
      }
      for (; k <= kin1; ++k) row1(k, true);
      for (; k <= hi; ++k) row1(k, false);
      if (MODE == LM_STIFF) {
        T xq[P];
#pragma unroll
        for (int m = 0; m < P; ++m) xq[m] = T(0);
        auto back = [&](int k, T yk, const T* uk) {
          T x = yk;
#pragma unroll
          for (int e = 1; e <= P; ++e) x -= uk[e - 1] * xq[e - 1];
          if (FUSED) gdst[k * stride] = x;  // y / z lines: straight to global memory
          else col[k * LP] = x;
#pragma unroll
          for (int m = P - 1; m >= 1; --m) xq[m] = xq[m - 1];
          xq[0] = x;
        };
        k = hi;
        for (; k - 7 >= lo; k -= 8) {
          T yy[8], uu[8][P];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            yy[u] = col[(k - u) * LP];
#pragma unroll
            for (int e = 1; e <= P; ++e) uu[u][e - 1] = su[(e - 1) * plane + (k - u) * LP + t];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) back(k - u, yy[u], uu[u]);
        }
        for (; k >= lo; --k) {
          T uk[P];
#pragma unroll
          for (int e = 1; e <= P; ++e) uk[e - 1] = su[(e - 1) * plane + k * LP + t];
          back(k, col[k * LP], uk);
        }
      }
    } else {
      const int f = dch ? 1 : 0;
      // LM_DERIV: the right-hand side of row k is (A u)_k; a register window
      // keeps u[k-P .. k+P] because col[k] is overwritten by the elimination.
      T win[W];
      if (MODE == LM_DERIV) {
#pragma unroll
        for (int d = 0; d < W; ++d) {
          const int j = lo + d - P;
          win[d] = (j >= 0 && j < N) ? col[j * LP] : T(0);
        }
      }
      T yq[P];
#pragma unroll
      for (int m = 0; m < P; ++m) yq[m] = T(0);
      // forward row k; CONST: factors (and A) are the mid-line constants
      // rk: r[k] (MASS) or u[k + P + 1] (DERIV), loaded by the caller
      auto fwd = [&](int k, bool cst, T rk) {
        const T* tb = tab + k * TABW;
        T y;
        if (MODE == LM_DERIV) {
          const T nxt = rk;
          y = T(0);
#pragma unroll
          for (int d = 0; d < W; ++d) y += (cst ? ax.inner[OP_A][d] : tb[3 * P + 1 + d]) * win[d];
#pragma unroll
          for (int d = 0; d < W - 1; ++d) win[d] = win[d + 1];
          win[W - 1] = nxt;
        } else {
          y = rk;
        }
#pragma unroll
        for (int m = 1; m <= P; ++m) y -= (cst ? ax.luc[f][m - 1] : tb[m - 1]) * yq[m - 1];
        col[k * LP] = y;
#pragma unroll
        for (int m = P - 1; m >= 1; --m) yq[m] = yq[m - 1];
        yq[0] = y;
      };
      int c0 = max(lo, ax.lu_lo[f]), c1 = min(hi, ax.lu_hi[f]);
      if (MODE == LM_DERIV) {
        c0 = max(c0, ax.inner_lo);
        c1 = min(c1, ax.inner_hi);
      }
      auto ld = [&](int k) -> T {
        if (MODE == LM_DERIV) {
          const int j = k + P + 1;
          return j < N ? col[j * LP] : T(0);
        }
        return col[k * LP];
      };
      int k = lo;
      for (; k < c0 && k <= hi; ++k) fwd(k, false, ld(k));
      // constant rows in blocks of 8: all loads of a block precede its stores
      for (; k + 7 <= c1; k += 8) {
        T rr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) rr[u] = ld(k + u);
#pragma unroll
        for (int u = 0; u < 8; ++u) fwd(k + u, true, rr[u]);
      }
      for (; k <= c1; ++k) fwd(k, true, ld(k));
      for (; k <= hi; ++k) fwd(k, false, ld(k));
      T xq[P];
#pragma unroll
      for (int m = 0; m < P; ++m) xq[m] = T(0);
      auto bwd = [&](int k, bool cst, T yk) {
        const T* tb = tab + k * TABW;
        T x = (cst ? ax.luc[f][P] : tb[P]) * yk;
#pragma unroll
        for (int e = 1; e <= P; ++e) x -= (cst ? ax.luc[f][P + e] : tb[P + e]) * xq[e - 1];
        if (FUSED) {  // y / z lines: straight to global memory
          if (MODE == LM_DERIV) red_add(gdst + k * stride, job.scale * x);
          else gdst[k * stride] = x;
        } else {
          col[k * LP] = x;
        }
#pragma unroll
        for (int m = P - 1; m >= 1; --m) xq[m] = xq[m - 1];
        xq[0] = x;
      };
      const int b0 = max(lo, ax.lu_lo[f]), b1 = min(hi, ax.lu_hi[f]);
      k = hi;
      for (; k > b1; --k) bwd(k, false, col[k * LP]);
      for (; k - 7 >= b0; k -= 8) {
        T yy[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) yy[u] = col[(k - u) * LP];
#pragma unroll
        for (int u = 0; u < 8; ++u) bwd(k - u, true, yy[u]);
      }
      for (; k >= b0; --k) bwd(k, true, col[k * LP]);
      for (; k >= lo; --k) bwd(k, false, col[k * LP]);
    }
    if (FUSED) {
      if (MODE != LM_DERIV) {  // fixed coefficients
        for (int k = 0; k < lo; ++k) gdst[k * stride] = T(0);
        for (int k = hi + 1; k < N; ++k) gdst[k * stride] = T(0);
      }
    } else {
      for (int k = 0; k < lo; ++k) col[k * LP] = T(0);
      for (int k = hi + 1; k < N; ++k) col[k * LP] = T(0);
    }
  }
  if (FUSED) return;  // y / z results are already in global memory
  __syncthreads();

  // ---- write back (LM_DERIV: dst += scale * x, done by the L2)
  const T scale = job.scale;
  T* dst = job.dst;
  if (XDIR) {
    const long long b0 = (long long)L0 * lp.pitch;
    int line = 0;
    for (; line + 3 < cnt; line += 4) {  // four lines per batch: loads before stores
      T v[4][5];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const int k = t + q * LINES;
          v[u][q] = k < N ? sr[k * LP + line + u] : T(0);
        }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        T* g = dst + b0 + (long long)(line + u) * lp.pitch;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const int k = t + q * LINES;
          if (k < N) {
            if (MODE == LM_DERIV) red_add(g + k, scale * v[u][q]);
            else g[k] = v[u][q];
          }
        }
      }
      for (int k = t + 5 * LINES; k < N; k += LINES)  // lines longer than 5 * LINES
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          T* g = dst + b0 + (long long)(line + u) * lp.pitch;
          const T vv = sr[k * LP + line + u];
          if (MODE == LM_DERIV) red_add(g + k, scale * vv);
          else g[k] = vv;
        }
    }
    for (; line < cnt; ++line) {
      T* g = dst + b0 + (long long)line * lp.pitch;
      for (int k = t; k < N; k += LINES) {
        const T v = sr[k * LP + line];
        if (MODE == LM_DERIV) red_add(g + k, scale * v);
        else g[k] = v;
      }
    }
  } else if (t < cnt) {
    T* g = dst + off;
    const T* s = sr + t;
    int k = 0;
    for (; k + 7 < N; k += 8) {  // eight shared loads, then eight global stores
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = s[u * LP];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (MODE == LM_DERIV) red_add(g + u * stride, scale * v[u]);
        else g[u * stride] = v[u];
      }
      g += 8 * stride;
      s += 8 * LP;
    }
    for (; k < N; ++k) {
      if (MODE == LM_DERIV) red_add(g, scale * *s);
      else *g = *s;
      g += stride;
      s += LP;
    }
  }
}

// Streaming banded solves along y or z (Appendix, eqs. split1/split2): one
// thread per line, consecutive threads on consecutive x, so every row of a warp
// is one coalesced access; nothing is staged in shared memory, and the warps of
// a whole launch are resident at once.  The forward sweep writes y to dst (DERIV:
// to job.work) and the backward sweep reads it back through the L2.  Loads of
// the next block of rows are issued before the stores of the current block.
//   LM_STIFF: dst = (M + diag(c) S)^-1 src with the row factors precomputed per
//             dt by the LM_PIVOT pass (job.fac: multipliers, normalised upper
//             factors; job.aux2: inverse pivots).  This is the form launched.
//   LM_MASS : dst = M^-1 src, and LM_DERIV: dst += scale * M^-1 (A src), also
//             compile; launch_line keeps those lines on the staged kernel,
//             which measured faster for them (1 KB of intermediate per line of
//             a whole launch does not stay in L2).
template <typename T, int P, int MODE>
__global__ void __launch_bounds__(128) line_direct_kernel(const LineJobs<T> jobs, const LineParams lp,
                                                          const AxisDev<T> ax) {
  constexpr int W = 2 * P + 1;
  constexpr int B = 8;  // rows per block of loads
  const LineJob<T> job = blockIdx.y == 0 ? jobs.job[0] : (blockIdx.y == 1 ? jobs.job[1] : jobs.job[2]);
  const long long L = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= lp.nlines) return;
  long long off, stride;
  if (lp.dir == 1) {  // line L = z * N_x + x
    off = (L / lp.Nx) * (long long)lp.pitch * lp.Ny + (L % lp.Nx);
    stride = lp.pitch;
  } else {            // line L = y * N_x + x
    off = (L / lp.Nx) * (long long)lp.pitch + (L % lp.Nx);
    stride = (long long)lp.pitch * lp.Ny;
  }
  const int N = lp.N;
  const int dch = job.dirichlet;
  const int lo = dch ? 1 : 0, hi = dch ? N - 2 : N - 1;
  const int f = dch ? 1 : 0;
  const T* src = job.src + off;  // may alias dst (in-place solves)
  T* yv = (MODE == LM_DERIV ? job.work : job.dst) + off;

  // ---- forward sweep
  T yq[P];
#pragma unroll
  for (int m = 0; m < P; ++m) yq[m] = T(0);
  T win[W];  // DERIV: u[k-P .. k+P]
  if (MODE == LM_DERIV) {
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const int j = lo + d - P;
      win[d] = (j >= 0 && j < N) ? src[j * stride] : T(0);
    }
  }
  // right-hand side of row k: r[k] (MASS, STIFF) or u[k+P+1] (DERIV, window feed)
  auto ld = [&](int k) -> T {
    if (MODE == LM_DERIV) {
      const int j = k + P + 1;
      return j < N ? src[j * stride] : T(0);
    }
    return src[k * stride];
  };
  // one forward row; cst: mid-line constants (MASS, DERIV); lk: STIFF multipliers
  auto fwd = [&](int k, bool cst, T rk, const T* lk) {
    T y;
    if (MODE == LM_DERIV) {
      y = T(0);
#pragma unroll
      for (int d = 0; d < W; ++d) y += (cst ? ax.inner[OP_A][d] : ax.band[OP_A][k * W + d]) * win[d];
#pragma unroll
      for (int d = 0; d < W - 1; ++d) win[d] = win[d + 1];
      win[W - 1] = rk;
    } else {
      y = rk;
    }
#pragma unroll
    for (int m = 1; m <= P; ++m) {
      T lm;
      if (MODE == LM_STIFF) lm = lk[m - 1];
      else lm = cst ? ax.luc[f][m - 1] : ax.luL[f][k * P + m - 1];
      y -= lm * yq[m - 1];
    }
    yv[k * stride] = y;
#pragma unroll
    for (int m = P - 1; m >= 1; --m) yq[m] = yq[m - 1];
    yq[0] = y;
  };
  if (MODE == LM_STIFF) {
    int k = lo;
    if (k + B - 1 <= hi) {  // blocks of rows; the next block's loads precede this block's stores
      T rr[B], ll[B][P], rn[B], ln[B][P];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        rr[u] = src[(k + u) * stride];
#pragma unroll
        for (int m = 0; m < P; ++m) ll[u][m] = job.fac[m][off + (k + u) * stride];
      }
      for (; k + B - 1 <= hi; k += B) {
        const bool more = k + 2 * B - 1 <= hi;
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) {
            rn[u] = src[(k + B + u) * stride];
#pragma unroll
            for (int m = 0; m < P; ++m) ln[u][m] = job.fac[m][off + (k + B + u) * stride];
          }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) fwd(k + u, false, rr[u], ll[u]);
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) {
            rr[u] = rn[u];
#pragma unroll
            for (int m = 0; m < P; ++m) ll[u][m] = ln[u][m];
          }
        }
      }
    }
    for (; k <= hi; ++k) {
      T lk[P];
#pragma unroll
      for (int m = 0; m < P; ++m) lk[m] = job.fac[m][off + k * stride];
      fwd(k, false, src[k * stride], lk);
    }
  } else {
    int c0 = max(lo, ax.lu_lo[f]), c1 = min(hi, ax.lu_hi[f]);
    if (MODE == LM_DERIV) {
      c0 = max(c0, ax.inner_lo);
      c1 = min(c1, ax.inner_hi);
    }
    int k = lo;
    for (; k < c0 && k <= hi; ++k) fwd(k, false, ld(k), nullptr);
    if (k + B - 1 <= c1) {  // constant rows: the next block's loads precede this block's stores
      T cur[B], nxt[B];
#pragma unroll
      for (int u = 0; u < B; ++u) cur[u] = ld(k + u);
      for (; k + B - 1 <= c1; k += B) {
        const bool more = k + 2 * B - 1 <= c1;
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) nxt[u] = ld(k + B + u);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) fwd(k + u, true, cur[u], nullptr);
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) cur[u] = nxt[u];
        }
      }
    }
    for (; k <= c1; ++k) fwd(k, true, ld(k), nullptr);
    for (; k <= hi; ++k) fwd(k, false, ld(k), nullptr);
  }

  // ---- backward sweep
  T xq[P];
#pragma unroll
  for (int m = 0; m < P; ++m) xq[m] = T(0);
  const T scale = job.scale;
  T* out = job.dst + off;
  auto bwd = [&](int k, bool cst, T yk, T ik, const T* uk) {
    T x;
    if (MODE == LM_STIFF) {
      x = ik * yk;
#pragma unroll
      for (int e = 1; e <= P; ++e) x -= uk[e - 1] * xq[e - 1];
    } else {
      x = (cst ? ax.luc[f][P] : ax.luInv[f][k]) * yk;
#pragma unroll
      for (int e = 1; e <= P; ++e) x -= (cst ? ax.luc[f][P + e] : ax.luU[f][k * P + e - 1]) * xq[e - 1];
    }
    if (MODE == LM_DERIV) red_add(out + k * stride, scale * x);
    else out[k * stride] = x;
#pragma unroll
    for (int m = P - 1; m >= 1; --m) xq[m] = xq[m - 1];
    xq[0] = x;
  };
  if (MODE == LM_STIFF) {
    int k = hi;
    if (k - B + 1 >= lo) {
      T yy[B], ii[B], uu[B][P], yn[B], in_[B], un[B][P];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const long long g = off + (k - u) * stride;
        yy[u] = yv[(k - u) * stride];
        ii[u] = job.aux2[g];
#pragma unroll
        for (int e = 0; e < P; ++e) uu[u][e] = job.fac[P + e][g];
      }
      for (; k - B + 1 >= lo; k -= B) {
        const bool more = k - 2 * B + 1 >= lo;
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) {
            const long long g = off + (k - B - u) * stride;
            yn[u] = yv[(k - B - u) * stride];
            in_[u] = job.aux2[g];
#pragma unroll
            for (int e = 0; e < P; ++e) un[u][e] = job.fac[P + e][g];
          }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) bwd(k - u, false, yy[u], ii[u], uu[u]);
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) {
            yy[u] = yn[u];
            ii[u] = in_[u];
#pragma unroll
            for (int e = 0; e < P; ++e) uu[u][e] = un[u][e];
          }
        }
      }
    }
    for (; k >= lo; --k) {
      const long long g = off + k * stride;
      T uk[P];
#pragma unroll
      for (int e = 0; e < P; ++e) uk[e] = job.fac[P + e][g];
      bwd(k, false, yv[k * stride], job.aux2[g], uk);
    }
  } else {
    const int b0 = max(lo, ax.lu_lo[f]), b1 = min(hi, ax.lu_hi[f]);
    int k = hi;
    for (; k > b1; --k) bwd(k, false, yv[k * stride], T(0), nullptr);
    if (k - B + 1 >= b0) {
      T cur[B], nxt[B];
#pragma unroll
      for (int u = 0; u < B; ++u) cur[u] = yv[(k - u) * stride];
      for (; k - B + 1 >= b0; k -= B) {
        const bool more = k - 2 * B + 1 >= b0;
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) nxt[u] = yv[(k - B - u) * stride];
        }
#pragma unroll
        for (int u = 0; u < B; ++u) bwd(k - u, true, cur[u], T(0), nullptr);
        if (more) {
#pragma unroll
          for (int u = 0; u < B; ++u) cur[u] = nxt[u];
        }
      }
    }
    for (; k >= b0; --k) bwd(k, true, yv[k * stride], T(0), nullptr);
    for (; k >= lo; --k) bwd(k, false, yv[k * stride], T(0), nullptr);
  }
  if (MODE != LM_DERIV && dch) {  // fixed coefficients
    out[0] = T(0);
    out[(N - 1) * stride] = T(0);
  }
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Whole-line bulk copies (TMA, no tensor map): global -> shared completing on an
// mbarrier, shared -> global as a store or an FP32 add.  Addresses and sizes are
// multiples of 16 bytes.
__device__ __forceinline__ void xw_bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"((unsigned)__cvta_generic_to_shared(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void xw_bar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(float* smem, const float* gmem, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(bytes), "r"((unsigned)__cvta_generic_to_shared(bar))
               : "memory");
}
// the issuing thread's own shared writes before the copy (generic -> async proxy)
__device__ __forceinline__ void bulk_store(void* gmem, const void* smem, unsigned bytes, bool add) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (add)
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;\n" ::"l"(gmem),
                 "r"((unsigned)__cvta_generic_to_shared(smem)), "r"(bytes)
                 : "memory");
  else
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem),
                 "r"((unsigned)__cvta_generic_to_shared(smem)), "r"(bytes)
                 : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// shared memory may be released once the issuing thread's bulk stores have read it
__device__ __forceinline__ void bulk_store_drain() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// Wait for phase `parity` of the barrier with an iteration limit; false if it gave up.
__device__ __forceinline__ bool xw_bar_wait(unsigned long long* bar, unsigned parity, int budget = 1 << 22) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  for (int it = 0; it < budget; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Banded solves along x (rows contiguous in memory), one warp per 32 lines and
// no block-wide synchronisation (Appendix, eqs. split1/split2).  Each lane
// stages its line whole into shared memory as row [line][k] with one bulk copy
// (the row pitch lpk is a multiple of 4 with lpk / 4 odd, so the 16-byte
// accesses of eight lanes to eight lines fall into 32 distinct banks), runs
// the line's recurrence in place, four rows per shared access, and writes the
// row back with one bulk store (DERIV: a bulk FP32 add).  Rows are copied to
// the pitch (a multiple of 4): the padding of dst receives zeros (MASS) or an
// added zero (DERIV).
//   LM_MASS : dst = M^-1 src (full or Dirichlet-reduced mass LU)
//   LM_DERIV: dst += scale * M^-1 (A src) (the bulk add performs the update)
// Blocks of four rows whose factors (and A rows) all equal the mid-line
// constants use registers; the other rows read the 1D tables, whose rows in the
// constant range hold the same values.
template <int P, int MODE>
__global__ void __launch_bounds__(32) line_xw_kernel(const LineJobs<float> jobs, const LineParams lp,
                                                     const AxisDev<float> ax, int lpk) {
  constexpr int W = 2 * P + 1;
  extern __shared__ __align__(16) float xw_plane[];  // [32][lpk]
  const LineJob<float> job = blockIdx.y == 0 ? jobs.job[0] : (blockIdx.y == 1 ? jobs.job[1] : jobs.job[2]);
  const int lane = threadIdx.x;
  const long long L0 = (long long)blockIdx.x * 32;
  const int cnt = (int)min(32LL, lp.nlines - L0);
  const int N = lp.N, NC = (N + 3) >> 2;  // 16-byte chunks per line (the pitch holds 4 NC elements)
  const long long pitch = lp.pitch;

  __shared__ __align__(8) unsigned long long bar;
  // ---- stage: one bulk copy per line
  if (lane == 0) {
    xw_bar_init(&bar);
    xw_bar_expect(&bar, (unsigned)(cnt * 16 * NC));
  }
  __syncwarp();
  if (lane < cnt) bulk_load(xw_plane + lane * lpk, job.src + (L0 + lane) * pitch, 16u * NC, &bar);
  if (!xw_bar_wait(&bar, 0)) {  // give up: report, give the copies a bounded time, leave
    if (lane == 0) atomicOr(lp.err, 1);
    xw_bar_wait(&bar, 0);
    return;
  }

  if (lane < cnt) {
    float* row = xw_plane + lane * lpk;
    for (int k = N; k < lpk; ++k) row[k] = 0.f;  // pitch padding (and slack) reads as zeros
    const int dch = job.dirichlet;
    const int lo = dch ? 1 : 0, hi = dch ? N - 2 : N - 1;
    const int llo = dch ? ax.lu_lo[1] : ax.lu_lo[0], lhi = dch ? ax.lu_hi[1] : ax.lu_hi[0];
    const float* Lt = dch ? ax.luL[1] : ax.luL[0];
    const float* It = dch ? ax.luInv[1] : ax.luInv[0];
    const float* Ut = dch ? ax.luU[1] : ax.luU[0];
    const float* At = ax.band[OP_A];
    float lc[P], uc[P], ac[W];
#pragma unroll
    for (int m = 0; m < P; ++m) {
      lc[m] = dch ? ax.luc[1][m] : ax.luc[0][m];
      uc[m] = dch ? ax.luc[1][P + 1 + m] : ax.luc[0][P + 1 + m];
    }
    const float ic = dch ? ax.luc[1][P] : ax.luc[0][P];
#pragma unroll
    for (int d = 0; d < W; ++d) ac[d] = ax.inner[OP_A][d];
    int c0 = max(lo, llo), c1 = min(hi, lhi);
    if (MODE == LM_DERIV) {
      c0 = max(c0, ax.inner_lo);
      c1 = min(c1, ax.inner_hi);
    }

    // ---- forward sweep (DERIV: right-hand side (A u)_k from a window u[k-P .. k+P])
    float yq[P];
#pragma unroll
    for (int m = 0; m < P; ++m) yq[m] = 0.f;
    float win[W];
#pragma unroll
    for (int d = 0; d < W; ++d) win[d] = (MODE == LM_DERIV && d >= P && d - P < N) ? row[d - P] : 0.f;
    // registers hold rows k0 .. k0 + 4 NV - 1: the block and, for DERIV, the
    // window feed u[k + P + 1] of its last row (k0 + P + 4); one more block of 4
    // is loaded ahead, so lpk >= 4 NC + 4 NV (the launcher leaves 12 of slack)
    constexpr int NV = MODE == LM_DERIV ? (P + 8) / 4 : 1;
    float4 buf[NV + 1];
#pragma unroll
    for (int v = 0; v < NV; ++v) buf[v] = *reinterpret_cast<const float4*>(row + 4 * v);
    for (int b = 0; b < NC; ++b) {
      const int k0 = 4 * b;
      // the rows ahead are read before this block's results are stored
      buf[NV] = *reinterpret_cast<const float4*>(row + k0 + 4 * NV);
      float cur[4 * NV];  // DERIV: u[k0 .. k0 + 4 NV - 1]
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        cur[4 * v] = buf[v].x;
        cur[4 * v + 1] = buf[v].y;
        cur[4 * v + 2] = buf[v].z;
        cur[4 * v + 3] = buf[v].w;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) buf[v] = buf[v + 1];
      float out[4];
      if (k0 >= c0 && k0 + 3 <= c1) {  // constant block (warp-uniform)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float y;
          if (MODE == LM_DERIV) {
            y = 0.f;
#pragma unroll
            for (int d = 0; d < W; ++d) y += ac[d] * win[d];
#pragma unroll
            for (int d = 0; d < W - 1; ++d) win[d] = win[d + 1];
            win[W - 1] = cur[u + P + 1];
          } else {
            y = cur[u];
          }
#pragma unroll
          for (int m = P - 1; m >= 0; --m) y -= lc[m] * yq[m];  // nearest term last: one FMA per row on the chain
          out[u] = y;
#pragma unroll
          for (int m = P - 1; m >= 1; --m) yq[m] = yq[m - 1];
          yq[0] = y;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + u;
          const bool live = k >= lo && k <= hi;
          float y = 0.f;
          if (MODE == LM_DERIV) {
            if (live) {
#pragma unroll
              for (int d = 0; d < W; ++d) y += At[k * W + d] * win[d];
            }
#pragma unroll
            for (int d = 0; d < W - 1; ++d) win[d] = win[d + 1];
            win[W - 1] = cur[u + P + 1];
          } else {
            y = cur[u];
          }
          if (live) {
#pragma unroll
            for (int m = P - 1; m >= 0; --m) y -= Lt[k * P + m] * yq[m];
#pragma unroll
            for (int m = P - 1; m >= 1; --m) yq[m] = yq[m - 1];
            yq[0] = y;
          }
          out[u] = live ? y : 0.f;
        }
      }
      *reinterpret_cast<float4*>(row + k0) = make_float4(out[0], out[1], out[2], out[3]);
    }

    // ---- backward sweep
    const int b0 = max(lo, llo), b1 = min(hi, lhi);
    float xq[P];
#pragma unroll
    for (int m = 0; m < P; ++m) xq[m] = 0.f;
    float4 yv = *reinterpret_cast<const float4*>(row + 4 * (NC - 1));
    for (int b = NC - 1; b >= 0; --b) {
      const int k0 = 4 * b;
      const float yy[4] = {yv.x, yv.y, yv.z, yv.w};
      if (b > 0) yv = *reinterpret_cast<const float4*>(row + k0 - 4);  // next block ahead of the stores
      float out[4];
      if (k0 >= b0 && k0 + 3 <= b1) {
#pragma unroll
        for (int u = 3; u >= 0; --u) {
          float x = ic * yy[u];
#pragma unroll
          for (int e = P - 1; e >= 0; --e) x -= uc[e] * xq[e];
          out[u] = MODE == LM_DERIV ? job.scale * x : x;
#pragma unroll
          for (int m = P - 1; m >= 1; --m) xq[m] = xq[m - 1];
          xq[0] = x;
        }
      } else {
#pragma unroll
        for (int u = 3; u >= 0; --u) {
          const int k = k0 + u;
          if (k >= lo && k <= hi) {
            float x = It[k] * yy[u];
#pragma unroll
            for (int e = P - 1; e >= 0; --e) x -= Ut[k * P + e] * xq[e];
            out[u] = MODE == LM_DERIV ? job.scale * x : x;
#pragma unroll
            for (int m = P - 1; m >= 1; --m) xq[m] = xq[m - 1];
            xq[0] = x;
          } else {
            out[u] = 0.f;
          }
        }
      }
      *reinterpret_cast<float4*>(row + k0) = make_float4(out[0], out[1], out[2], out[3]);
    }
    // ---- write back (MASS: dst = x; DERIV: dst += scale * x, scaled above)
    bulk_store(job.dst + (L0 + lane) * pitch, row, 16u * NC, MODE == LM_DERIV);
    bulk_store_drain();
  }
}

// Stiffness solves along x (FP32), one warp per 32 lines, with the row factors
// of M + diag(c) S precomputed per dt by the LM_PIVOT pass (multipliers
// fac[0..P-1], normalised upper factors fac[P..2P-1], inverse pivots aux2):
//   forward  y_k = r_k - sum_m l_m[k] y_{k-m},
//   backward x_k = y_k / pivot_k - sum_e u_e[k] x_{k+e},   k in lo .. hi,
// the arithmetic of the streaming y / z form.  The right-hand side and y stay
// in shared memory as rows [line][k]; the factor rows stream through a
// two-stage ring of 16-row chunks (cp.async, one group per chunk), so the next
// chunk is in flight while this one is solved.  Each lane stores its row back
// with one bulk copy.
// four consecutive elements (16 bytes of FP32, 32 of FP64) from / to shared memory
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// factor rows per ring chunk: 32 (FP32), 16 (FP64, so that two warps fit per SM)
template <typename T>
__host__ __device__ constexpr int xws_rows() { return sizeof(T) == 4 ? 32 : 16; }
template <typename T, int P>
__global__ void __launch_bounds__(32) line_xws_kernel(const LineJobs<T> jobs, const LineParams lp, int lpk) {
  constexpr int CH = xws_rows<T>(), CHP = CH + 4, NA = P + 1;  // rows per chunk, chunk row pitch, arrays per stage
  constexpr int EP = 16 / sizeof(T), PPL = CH / EP;          // elements per 16-byte piece, pieces per chunk row
  static_assert(sizeof(T) != 4 || ((CHP / 4) & 1) == 1, "conflict-free 16-byte lane accesses");
  extern __shared__ __align__(16) unsigned char xs_raw[];
  T* plane = reinterpret_cast<T*>(xs_raw);  // [32][lpk]: r, then y, then x
  T* ring = plane + 32 * lpk;               // [2][NA][32][CHP]
  const LineJob<T> job = blockIdx.y == 0 ? jobs.job[0] : (blockIdx.y == 1 ? jobs.job[1] : jobs.job[2]);
  const int lane = threadIdx.x;
  const long long L0 = (long long)blockIdx.x * 32;
  const int cnt = (int)min(32LL, lp.nlines - L0);
  const int N = lp.N, N4 = (N + 3) & ~3, nch = (N + CH - 1) / CH;
  const long long pitch = lp.pitch, base = L0 * pitch;
  const int dch = job.dirichlet;
  const int lo = dch ? 1 : 0, hi = dch ? N - 2 : N - 1;
  auto slot = [&](int st, int a, int i) { return ring + ((st * NA + a) * 32 + i) * CHP; };
  // chunk ch: 32 lines x PPL pieces of 16 bytes
  auto issue = [&](int ch, int st, bool fwd) {
    const int k0 = ch * CH;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
      const int t = q * 32 + lane, i = t / PPL, j = t % PPL, k = k0 + EP * j;
      if (i < cnt && k < N4) {
        const long long g = base + i * pitch + k;
        if (fwd) {
          cp_async16(plane + i * lpk + k, job.src + g);
#pragma unroll
          for (int m = 0; m < P; ++m) cp_async16(slot(st, m, i) + EP * j, job.fac[m] + g);
        } else {
          cp_async16(slot(st, 0, i) + EP * j, job.aux2 + g);
#pragma unroll
          for (int e = 0; e < P; ++e) cp_async16(slot(st, 1 + e, i) + EP * j, job.fac[P + e] + g);
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  T* row = plane + lane * lpk;
  const bool mine = lane < cnt;

  // ---- forward sweep
  T yq[P];
#pragma unroll
  for (int m = 0; m < P; ++m) yq[m] = T(0);
  issue(0, 0, true);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) {
      issue(ch + 1, (ch + 1) & 1, true);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncwarp();
    if (mine) {
      const int st = ch & 1;
#pragma unroll
      for (int bb = 0; bb < CH / 4; ++bb) {
        const int k0 = ch * CH + 4 * bb;
        if (k0 >= N4) break;
        T r[4], l[P][4], out[4];
        ld4(row + k0, r);
#pragma unroll
        for (int m = 0; m < P; ++m) ld4(slot(st, m, lane) + 4 * bb, l[m]);
        const bool all = k0 >= lo && k0 + 3 <= hi;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool live = all || (k0 + u >= lo && k0 + u <= hi);
          T y = r[u];
#pragma unroll
          for (int m = P - 1; m >= 0; --m) y -= l[m][u] * yq[m];
          if (live) {
#pragma unroll
            for (int m = P - 1; m >= 1; --m) yq[m] = yq[m - 1];
            yq[0] = y;
          }
          out[u] = live ? y : T(0);
        }
        st4(row + k0, out);
      }
    }
    __syncwarp();  // this stage is refilled two chunks on
  }

  // ---- backward sweep
  T xq[P];
#pragma unroll
  for (int m = 0; m < P; ++m) xq[m] = T(0);
  issue(nch - 1, (nch - 1) & 1, false);
  for (int ch = nch - 1; ch >= 0; --ch) {
    if (ch > 0) {
      issue(ch - 1, (ch - 1) & 1, false);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncwarp();
    if (mine) {
      const int st = ch & 1;
#pragma unroll
      for (int bb = CH / 4 - 1; bb >= 0; --bb) {
        const int k0 = ch * CH + 4 * bb;
        if (k0 >= N4) continue;
        T y[4], inv[4], uu[P][4], out[4];
        ld4(row + k0, y);
        ld4(slot(st, 0, lane) + 4 * bb, inv);
#pragma unroll
        for (int e = 0; e < P; ++e) ld4(slot(st, 1 + e, lane) + 4 * bb, uu[e]);
        const bool all = k0 >= lo && k0 + 3 <= hi;
#pragma unroll
        for (int u = 3; u >= 0; --u) {
          const bool live = all || (k0 + u >= lo && k0 + u <= hi);
          T x = inv[u] * y[u];
#pragma unroll
          for (int e = P - 1; e >= 0; --e) x -= uu[e][u] * xq[e];
          if (live) {
#pragma unroll
            for (int m = P - 1; m >= 1; --m) xq[m] = xq[m - 1];
            xq[0] = x;
          }
          out[u] = live ? x : T(0);
        }
        st4(row + k0, out);
      }
    }
    __syncwarp();
  }

  // ---- write back: one bulk store per line (rows to the pitch; zeros outside lo .. hi)
  if (mine) {
    bulk_store(job.dst + base + lane * pitch, row, (unsigned)(sizeof(T) * N4), false);
    bulk_store_drain();
  }
}

// ------------------------------------------------- E right-hand side (v2)
// One CTA per 32 x 8 x 8 output tile (256 threads).  For each of the six input
// fields a (8+2P) x (8+2P) x (32+2P) tile with halo is staged by cp.async
// (double buffered across fields) and contracted by sum factorisation: a z pass
// (thread per haloed (y,x) column, 8 outputs from a register window), a y pass
// (thread per (z',x) column) and an x pass (thread per two x outputs in four
// (z',y) rows), accumulating the a-, b- and c-scaled terms into registers.
// Each field enters exactly two terms of eq. (dupa1ab) (half step 1) or of its
// half-step-2 analogue (R2 instead of R1); the term plan is a compile-time
// table, so interior stencils are constant operands.  Rows near the boundary
// (outside 2p .. N-1-2p) read their band rows from the tables instead.
namespace rhs2 {
#ifndef ADI_RHS_NT
#define ADI_RHS_NT 256
#endif
#ifndef ADI_RHS_NBUF
#define ADI_RHS_NBUF 2
#endif
#ifndef ADI_RHS_MINB
#define ADI_RHS_MINB 2
#endif
constexpr int TX = 32, TY = 8, TZ = 8, NT = ADI_RHS_NT;  // compile-time tile and launch shape
constexpr int RG = NT / 16;                // x-pass row groups: 16 threads x 2 outputs cover a row of 32
constexpr int RPT = TZ * TY / RG;          // (z', y) rows per thread in the x pass

// the two terms of field F in half step H: ops per axis, output, coefficient, sign
template <int H, int F>
struct Plan;
#define ADI_PLAN(H, F, X0, Y0, Z0, O0, C0, S0, X1, Y1, Z1, O1, C1, S1)                   \
  template <>                                                                             \
  struct Plan<H, F> {                                                                     \
    static constexpr int x0 = X0, y0 = Y0, z0 = Z0, o0 = O0, c0 = C0;                     \
    static constexpr int x1 = X1, y1 = Y1, z1 = Z1, o1 = O1, c1 = C1;                     \
    static constexpr float s0 = S0, s1 = S1;                                              \
  };
// E1: a M(x)M(x)M E1 ; R1[3][1] = B(x)M(x)A -> E3 (c) ; R2[2][1] = B(x)A(x)M -> E2 (c)
ADI_PLAN(1, 0, OP_M, OP_M, OP_M, 0, CF_A, 1.f, OP_B, OP_M, OP_A, 2, CF_C, 1.f)
ADI_PLAN(2, 0, OP_M, OP_M, OP_M, 0, CF_A, 1.f, OP_B, OP_A, OP_M, 1, CF_C, 1.f)
// E2: a MMM E2 ; R1[1][2] = A(x)B(x)M -> E1 ; R2[3][2] = M(x)B(x)A -> E3
ADI_PLAN(1, 1, OP_M, OP_M, OP_M, 1, CF_A, 1.f, OP_A, OP_B, OP_M, 0, CF_C, 1.f)
ADI_PLAN(2, 1, OP_M, OP_M, OP_M, 1, CF_A, 1.f, OP_M, OP_B, OP_A, 2, CF_C, 1.f)
// E3: a MMM E3 ; R1[2][3] = M(x)A(x)B -> E2 ; R2[1][3] = A(x)M(x)B -> E1
ADI_PLAN(1, 2, OP_M, OP_M, OP_M, 2, CF_A, 1.f, OP_M, OP_A, OP_B, 1, CF_C, 1.f)
ADI_PLAN(2, 2, OP_M, OP_M, OP_M, 2, CF_A, 1.f, OP_A, OP_M, OP_B, 0, CF_C, 1.f)
// curl H = (C1 - C2) H scaled by b (both half steps):
// H1: +d3 H1 -> E2, -d2 H1 -> E3 ; H2: -d3 H2 -> E1, +d1 H2 -> E3 ; H3: +d2 H3 -> E1, -d1 H3 -> E2
ADI_PLAN(1, 3, OP_M, OP_M, OP_A, 1, CF_B, 1.f, OP_M, OP_A, OP_M, 2, CF_B, -1.f)
ADI_PLAN(2, 3, OP_M, OP_M, OP_A, 1, CF_B, 1.f, OP_M, OP_A, OP_M, 2, CF_B, -1.f)
ADI_PLAN(1, 4, OP_M, OP_M, OP_A, 0, CF_B, -1.f, OP_A, OP_M, OP_M, 2, CF_B, 1.f)
ADI_PLAN(2, 4, OP_M, OP_M, OP_A, 0, CF_B, -1.f, OP_A, OP_M, OP_M, 2, CF_B, 1.f)
ADI_PLAN(1, 5, OP_M, OP_A, OP_M, 0, CF_B, 1.f, OP_A, OP_M, OP_M, 1, CF_B, -1.f)
ADI_PLAN(2, 5, OP_M, OP_A, OP_M, 0, CF_B, 1.f, OP_A, OP_M, OP_M, 1, CF_B, -1.f)
#undef ADI_PLAN

__host__ __device__ constexpr int sidx(int op) { return op == OP_M ? 0 : (op == OP_A ? 1 : 2); }

// band value X[r][q] of op on axis D: interior rows use the constant stencil
template <typename T, int P, int D, int OP, bool INNER>
__device__ __forceinline__ T bandv(const RhsParams<T>& prm, int r, int q) {
  if (INNER) return prm.st[D].w[sidx(OP)][q];
  return prm.ax[D].band[OP][r * (2 * P + 1) + q];
}

template <typename T, int P>
struct Smem {
  static constexpr int HX = TX + 2 * P, HY = TY + 2 * P, HZ = TZ + 2 * P;
  static constexpr int BX = 40;       // tile row: x0-4 .. x0+35 (TMA box)
  static constexpr int XOFF = 4 - P;  // position of x0-P inside a tile row
  // row pitch of the y-pass results: odd (bank-conflict free scalar x pass), or
  // even for p = 2, whose passes move pairs of columns (8- / 16-byte accesses)
  static constexpr int HXP = P == 2 ? HX + 2 : HX + 1;
  // plane strides of the z- and y-pass results (SZ per z' of [y'][x'], SY per z'
  // of [y][x']); p = 2 pads both to 4 (mod 32) banks, so a half-warp of pair
  // accesses that straddles two planes touches 32 distinct banks
  static constexpr int SZ = P == 2 ? HY * HX + ((36 - (HY * HX) % 32) % 32) : HY * HX;
  static constexpr int SY = P == 2 ? TY * HXP + ((36 - (TY * HXP) % 32) % 32) : TY * HXP;
  static constexpr int TILE = HZ * HY * BX, ZR = TZ * SZ, YR = TZ * SY;
  // dynamic shared memory: 128 bytes of alignment slack, the tiles (TMA
  // destinations, 128-byte aligned), the pass buffers, then two mbarriers
  // band rows of the tile's output rows along z and y for tiles that reach a
  // boundary row: [op M, A, B][row][q], rows padded to WP (16-byte vectors)
  static constexpr int WP = (2 * P + 1 + 3) / 4 * 4;
  static constexpr int BT = 3 * (TZ + TY) * WP;
  static constexpr size_t DATA2 = sizeof(T) * (2 * (size_t)TILE + 2 * (size_t)ZR + 2 * (size_t)YR + BT);
  static constexpr int NBUF = (ADI_RHS_NBUF == 2 && DATA2 + 128 + 16 <= 227 * 1024) ? 2 : 1;  // double-buffer if it fits
  static constexpr size_t DATA = sizeof(T) * (NBUF * (size_t)TILE + 2 * (size_t)ZR + 2 * (size_t)YR + BT);
  static constexpr size_t BYTES = 128 + DATA + 16;
};

// the W band values of one staged row (16-byte vector loads from shared memory)
template <typename T, int W, int WP>
__device__ __forceinline__ void ldrow(const T* p, T (&r)[W]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < WP / 4; ++k) {
      const float4 v = reinterpret_cast<const float4*>(p)[k];
      const T e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * k + j < W) r[4 * k + j] = e[j];
    }
  } else {
#pragma unroll
    for (int k = 0; k < WP / 2; ++k) {
      const double2 v = reinterpret_cast<const double2*>(p)[k];
      if (2 * k < W) r[2 * k] = v.x;
      if (2 * k + 1 < W) r[2 * k + 1] = v.y;
    }
  }
}

// z pass: column i = (yy, xx) of the haloed plane, 8 outputs from a window of HZ values
template <typename T, int P, int OP, bool INNER>
__device__ __forceinline__ void zpass(const RhsParams<T>& prm, const T* tl, T* zr, const T* tz, int i) {
  using S = Smem<T, P>;
  constexpr int W = 2 * P + 1;
  const T* col = tl + (i / S::HX) * S::BX + S::XOFF + (i % S::HX);
  T w[S::HZ];
#pragma unroll
  for (int k = 0; k < S::HZ; ++k) w[k] = col[k * S::HY * S::BX];
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz) {
    T c[W];
    if (INNER) {
#pragma unroll
      for (int q = 0; q < W; ++q) c[q] = prm.st[2].w[sidx(OP)][q];
    } else {
      ldrow<T, W, S::WP>(tz + (sidx(OP) * TZ + zz) * S::WP, c);
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < W; ++q) s += c[q] * w[zz + q];
    zr[zz * S::SZ + i] = s;
  }
}

// y pass: column (zz, xx), 8 outputs from a window of HY values
template <typename T, int P, int OP, bool INNER>
__device__ __forceinline__ void yapply(const RhsParams<T>& prm, const T (&w)[Smem<T, P>::HY], T* yr, const T* ty, int zz,
                                       int xx) {
  using S = Smem<T, P>;
  constexpr int W = 2 * P + 1;
#pragma unroll
  for (int yy = 0; yy < TY; ++yy) {
    T c[W];
    if (INNER) {
#pragma unroll
      for (int q = 0; q < W; ++q) c[q] = prm.st[1].w[sidx(OP)][q];
    } else {
      ldrow<T, W, S::WP>(ty + (sidx(OP) * TY + yy) * S::WP, c);
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < W; ++q) s += c[q] * w[yy + q];
    yr[zz * S::SY + yy * S::HXP + xx] = s;
  }
}

template <typename T, int P>
__device__ __forceinline__ void yload(const T* zr, int zz, int xx, T (&w)[Smem<T, P>::HY]) {
  using S = Smem<T, P>;
  const T* src = zr + zz * S::SZ + xx;
#pragma unroll
  for (int k = 0; k < S::HY; ++k) w[k] = src[k * S::HX];
}

// x pass for two consecutive x outputs in four rows; adds coef * sign * value
template <typename T, int P, int OP, bool INNER, int OUT, int CK>
__device__ __forceinline__ void xpass(const RhsParams<T>& prm, const T* yr, int gx, int xp, int rg, float sg,
                                      T (&cf)[3][RPT][2], T (&acc)[3][RPT][2]) {
  using S = Smem<T, P>;
  constexpr int W = 2 * P + 1;
  T bx[2][W];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < W; ++q) bx[j][q] = bandv<T, P, 0, OP, INNER>(prm, min(gx + j, prm.Nx - 1), q);
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = r * RG + rg;  // half-warps read adjacent rows
    const T* src = yr + (row / TY) * S::SY + (row % TY) * S::HXP + xp;
    T w[W + 1];
#pragma unroll
    for (int q = 0; q < W + 1; ++q) w[q] = src[q];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < W; ++q) s += bx[j][q] * w[j + q];
      acc[OUT][r][j] += (T(sg) * cf[CK][r][j]) * s;
    }
  }
}

// ---- p = 2: passes on pairs of adjacent columns (two-element vector loads and
// stores, half the shared-memory instructions and address arithmetic per output)
template <typename T>
struct V2;
template <>
struct V2<float> {
  using t = float2;
};
template <>
struct V2<double> {
  using t = double2;
};

// z pass of column pair i2 = (yy, xx/2) for one or two z operators (ZSHARE: one)
template <typename T, int P, int OP0, int OP1, bool ZSHARE, bool INNER>
__device__ __forceinline__ void zpass2(const RhsParams<T>& prm, const T* tl, T* zr0, T* zr1, const T* tz, int i2) {
  using S = Smem<T, P>;
  using v2 = typename V2<T>::t;
  constexpr int W = 2 * P + 1;
  // pairs 0..15 of every row first (a half-warp reads 32 consecutive floats of
  // one tile row), then the remaining pairs of every row
  constexpr int NPR = S::HX / 2, NR = NPR - 16;
  static_assert(NR > 0, "a tile row holds more than 16 column pairs");
  const int j = i2 - S::HY * 16;
  const int yy = j < 0 ? i2 >> 4 : j / NR, xx = 2 * (j < 0 ? i2 & 15 : 16 + j % NR);
  const T* col = tl + yy * S::BX + S::XOFF + xx;
  v2 w[S::HZ];
#pragma unroll
  for (int k = 0; k < S::HZ; ++k) w[k] = *reinterpret_cast<const v2*>(col + k * S::HY * S::BX);
  const int o = yy * S::HX + xx;
#pragma unroll
  for (int zz = 0; zz < TZ; ++zz) {
    T cr[W], dr[W];
    if (INNER) {
#pragma unroll
      for (int q = 0; q < W; ++q) {
        cr[q] = prm.st[2].w[sidx(OP0)][q];
        dr[q] = prm.st[2].w[sidx(OP1)][q];
      }
    } else {
      ldrow<T, W, S::WP>(tz + (sidx(OP0) * TZ + zz) * S::WP, cr);
      if (!ZSHARE) ldrow<T, W, S::WP>(tz + (sidx(OP1) * TZ + zz) * S::WP, dr);
    }
    T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const T c = cr[q];
      a0 += c * w[zz + q].x;
      a1 += c * w[zz + q].y;
      if (!ZSHARE) {
        const T d = dr[q];
        b0 += d * w[zz + q].x;
        b1 += d * w[zz + q].y;
      }
    }
    v2 ra, rb;
    ra.x = a0;
    ra.y = a1;
    *reinterpret_cast<v2*>(zr0 + zz * S::SZ + o) = ra;
    if (!ZSHARE) {
      rb.x = b0;
      rb.y = b1;
      *reinterpret_cast<v2*>(zr1 + zz * S::SZ + o) = rb;
    }
  }
}

// y pass of column pair i2 = (zz, xx/2) for the field's two y operators
template <typename T, int P, int OP0, int OP1, bool ZSHARE, bool INNER>
__device__ __forceinline__ void ypass2(const RhsParams<T>& prm, const T* zr0, const T* zr1, T* yr0, T* yr1,
                                       const T* ty, int i2) {
  using S = Smem<T, P>;
  using v2 = typename V2<T>::t;
  constexpr int W = 2 * P + 1;
  const int zz = i2 / (S::HX / 2), xx = 2 * (i2 % (S::HX / 2));
  v2 w0[S::HY], w1[S::HY];
#pragma unroll
  for (int k = 0; k < S::HY; ++k) {
    w0[k] = *reinterpret_cast<const v2*>(zr0 + zz * S::SZ + k * S::HX + xx);
    w1[k] = ZSHARE ? w0[k] : *reinterpret_cast<const v2*>(zr1 + zz * S::SZ + k * S::HX + xx);
  }
#pragma unroll
  for (int yy = 0; yy < TY; ++yy) {
    T cr[W], dr[W];
    if (INNER) {
#pragma unroll
      for (int q = 0; q < W; ++q) {
        cr[q] = prm.st[1].w[sidx(OP0)][q];
        dr[q] = prm.st[1].w[sidx(OP1)][q];
      }
    } else {
      ldrow<T, W, S::WP>(ty + (sidx(OP0) * TY + yy) * S::WP, cr);
      ldrow<T, W, S::WP>(ty + (sidx(OP1) * TY + yy) * S::WP, dr);
    }
    T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const T c = cr[q];
      const T d = dr[q];
      a0 += c * w0[yy + q].x;
      a1 += c * w0[yy + q].y;
      b0 += d * w1[yy + q].x;
      b1 += d * w1[yy + q].y;
    }
    v2 ra, rb;
    ra.x = a0;
    ra.y = a1;
    rb.x = b0;
    rb.y = b1;
    *reinterpret_cast<v2*>(yr0 + zz * S::SY + yy * S::HXP + xx) = ra;
    *reinterpret_cast<v2*>(yr1 + zz * S::SY + yy * S::HXP + xx) = rb;
  }
}

// x pass as xpass, with the six-value windows read as three pairs
template <typename T, int P, int OP, bool INNER, int OUT, int CK>
__device__ __forceinline__ void xpass2(const RhsParams<T>& prm, const T* yr, int gx, int xp, int rg, float sg,
                                       T (&cf)[3][RPT][2], T (&acc)[3][RPT][2]) {
  using S = Smem<T, P>;
  using v2 = typename V2<T>::t;
  constexpr int W = 2 * P + 1;
  T bx[2][W];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < W; ++q) bx[j][q] = bandv<T, P, 0, OP, INNER>(prm, min(gx + j, prm.Nx - 1), q);
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = r * RG + rg;
    const T* src = yr + (row / TY) * S::SY + (row % TY) * S::HXP + xp;
    T w[W + 1];
#pragma unroll
    for (int q = 0; q < (W + 1) / 2; ++q) {
      const v2 u = *reinterpret_cast<const v2*>(src + 2 * q);
      w[2 * q] = u.x;
      w[2 * q + 1] = u.y;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < W; ++q) s += bx[j][q] * w[j + q];
      acc[OUT][r][j] += (T(sg) * cf[CK][r][j]) * s;
    }
  }
}

// TMA: one 3D box per field tile; x starts at x0 - 4 so that x * sizeof(T) is a
// multiple of 16 bytes; out-of-domain elements arrive as zeros.
constexpr int BOXX = 40;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
}

template <typename T, int P>
__device__ __forceinline__ void tma_tile(const CUtensorMap* map, T* dst, unsigned long long* bar, int x, int y, int z) {
  using S = Smem<T, P>;
  constexpr unsigned bytes = BOXX * S::HY * S::HZ * sizeof(T);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Wait for phase `parity` of the barrier with an iteration limit; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int budget = 1 << 22) {
  const unsigned a = smem_addr(bar);
  for (int it = 0; it < budget; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// The passes of one field, as three stages.  The kernel software-pipelines
// them across fields: [z(F) and x(F-1)] | [y(F)], so each field costs two
// block barriers (plus its tile wait) instead of three.
// Stage z: wait for the field's tile (every thread; the give-up decision is
// block-wide), z pass into s_zr.
template <typename T, int P, int H, int F>
__device__ __forceinline__ bool zstage(const RhsParams<T>& prm, T* s_tile, T* s_zr, unsigned long long* bars,
                                       const T* tz, bool inZ) {
  using S = Smem<T, P>;
  using PL = Plan<H, F>;
  const int tid = threadIdx.x;
  constexpr int B = S::NBUF == 2 ? (F & 1) : 0;                 // buffer of this field
  constexpr unsigned PAR = S::NBUF == 2 ? (F / 2) & 1 : F & 1;  // its barrier phase
  if (!__syncthreads_and(mbar_wait(&bars[B], PAR))) return false;
  const T* tl = s_tile + B * S::TILE;
  constexpr bool zshare = PL::z0 == PL::z1;
  if constexpr (P == 2) {  // pairs of columns
    for (int i2 = tid; i2 < S::HY * S::HX / 2; i2 += NT) {
      if (inZ) zpass2<T, P, PL::z0, PL::z1, zshare, true>(prm, tl, s_zr, s_zr + S::ZR, tz, i2);
      else zpass2<T, P, PL::z0, PL::z1, zshare, false>(prm, tl, s_zr, s_zr + S::ZR, tz, i2);
    }
  } else {  // p = 1, 3: one column per thread
    for (int i = tid; i < S::HY * S::HX; i += NT) {
      if (inZ) zpass<T, P, PL::z0, true>(prm, tl, s_zr, tz, i);
      else zpass<T, P, PL::z0, false>(prm, tl, s_zr, tz, i);
      if (!zshare) {
        if (inZ) zpass<T, P, PL::z1, true>(prm, tl, s_zr + S::ZR, tz, i);
        else zpass<T, P, PL::z1, false>(prm, tl, s_zr + S::ZR, tz, i);
      }
    }
  }
  return true;
}

// Stage y: s_zr -> s_yr for the field's two y operators.
template <typename T, int P, int H, int F>
__device__ __forceinline__ void ystage(const RhsParams<T>& prm, const T* s_zr, T* s_yr, const T* ty, bool inY) {
  using S = Smem<T, P>;
  using PL = Plan<H, F>;
  const int tid = threadIdx.x;
  constexpr bool zshare = PL::z0 == PL::z1;
  if constexpr (P == 2) {
    for (int i2 = tid; i2 < TZ * S::HX / 2; i2 += NT) {
      if (inY) ypass2<T, P, PL::y0, PL::y1, zshare, true>(prm, s_zr, s_zr + S::ZR, s_yr, s_yr + S::YR, ty, i2);
      else ypass2<T, P, PL::y0, PL::y1, zshare, false>(prm, s_zr, s_zr + S::ZR, s_yr, s_yr + S::YR, ty, i2);
    }
  } else {
    for (int i = tid; i < TZ * S::HX; i += NT) {
      const int zz = i / S::HX, xx = i % S::HX;
      T w[S::HY];
      yload<T, P>(s_zr, zz, xx, w);
      if (inY) yapply<T, P, PL::y0, true>(prm, w, s_yr, ty, zz, xx);
      else yapply<T, P, PL::y0, false>(prm, w, s_yr, ty, zz, xx);
      if (!zshare) yload<T, P>(s_zr + S::ZR, zz, xx, w);
      if (inY) yapply<T, P, PL::y1, true>(prm, w, s_yr + S::YR, ty, zz, xx);
      else yapply<T, P, PL::y1, false>(prm, w, s_yr + S::YR, ty, zz, xx);
    }
  }
}

// Stage x: s_yr -> the field's two terms accumulated into the output registers.
template <typename T, int P, int H, int F>
__device__ __forceinline__ void xstage(const RhsParams<T>& prm, const T* s_yr, int x0, bool inX, int xp, int rg,
                                       T (&cf)[3][RPT][2], T (&acc)[3][RPT][2]) {
  using S = Smem<T, P>;
  using PL = Plan<H, F>;
  const int gx = x0 + xp;  // band rows are clamped per output inside the x pass
  if constexpr (P == 2) {
    if (inX) {
      xpass2<T, P, PL::x0, true, PL::o0, PL::c0 - CF_A>(prm, s_yr, gx, xp, rg, PL::s0, cf, acc);
      xpass2<T, P, PL::x1, true, PL::o1, PL::c1 - CF_A>(prm, s_yr + S::YR, gx, xp, rg, PL::s1, cf, acc);
    } else {
      xpass2<T, P, PL::x0, false, PL::o0, PL::c0 - CF_A>(prm, s_yr, gx, xp, rg, PL::s0, cf, acc);
      xpass2<T, P, PL::x1, false, PL::o1, PL::c1 - CF_A>(prm, s_yr + S::YR, gx, xp, rg, PL::s1, cf, acc);
    }
  } else {
    if (inX) {
      xpass<T, P, PL::x0, true, PL::o0, PL::c0 - CF_A>(prm, s_yr, gx, xp, rg, PL::s0, cf, acc);
      xpass<T, P, PL::x1, true, PL::o1, PL::c1 - CF_A>(prm, s_yr + S::YR, gx, xp, rg, PL::s1, cf, acc);
    } else {
      xpass<T, P, PL::x0, false, PL::o0, PL::c0 - CF_A>(prm, s_yr, gx, xp, rg, PL::s0, cf, acc);
      xpass<T, P, PL::x1, false, PL::o1, PL::c1 - CF_A>(prm, s_yr + S::YR, gx, xp, rg, PL::s1, cf, acc);
    }
  }
}

// Field F of the pipeline: prefetch tile F+1, [z(F) and x(F-1)], y(F).  The
// tile buffer refilled here held field F-1, whose z pass ended before the
// previous barrier (one buffer: the tile is reloaded after z(F)); x(F-1) reads
// s_yr, which y(F) overwrites only after the barrier that follows it.
template <typename T, int P, int H, int F>
__device__ __forceinline__ bool pipe_field(const RhsParams<T>& prm, const TmaMaps& maps, T* s_tile, T* s_zr,
                                           T* s_yr, const T* s_bt, unsigned long long* bars, int x0, int y0, int z0, bool inZ,
                                           bool inY, bool inX, int xp, int rg, T (&cf)[3][RPT][2],
                                           T (&acc)[3][RPT][2]) {
  using S = Smem<T, P>;
  const int tid = threadIdx.x;
  if (S::NBUF == 2 && F + 1 < 6 && tid == 0)
    tma_tile<T, P>(&maps.m[F + 1], s_tile + ((F + 1) & 1) * S::TILE, &bars[(F + 1) & 1], x0 - 4, y0 - P, z0 - P);
  if (!zstage<T, P, H, F>(prm, s_tile, s_zr, bars, s_bt, inZ)) return false;
  if (F > 0) xstage<T, P, H, (F > 0 ? F - 1 : 0)>(prm, s_yr, x0, inX, xp, rg, cf, acc);
  __syncthreads();
  if (S::NBUF == 1 && F + 1 < 6 && tid == 0)  // single buffer (FP64): load the next tile during the y pass
    tma_tile<T, P>(&maps.m[F + 1], s_tile, &bars[0], x0 - 4, y0 - P, z0 - P);
  ystage<T, P, H, F>(prm, s_zr, s_yr, s_bt + 3 * TZ * S::WP, inY);
  __syncthreads();
  return true;
}
}  // namespace rhs2

template <typename T, int P, int H>
__global__ void __launch_bounds__(rhs2::NT, sizeof(T) == 4 ? ADI_RHS_MINB : 1)
    rhs_e_kernel(const RhsParams<T> prm, const __grid_constant__ TmaMaps maps) {
  using namespace rhs2;
  using S = Smem<T, P>;
  extern __shared__ __align__(128) unsigned char rhs_smem[];
  // TMA writes need a 128-byte aligned shared address: align at run time
  unsigned char* sbase = rhs_smem + ((128u - (smem_addr(rhs_smem) & 127u)) & 127u);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(sbase + S::DATA);  // 8-byte aligned
  T* s_tile = reinterpret_cast<T*>(sbase);     // NBUF x TILE (TMA destinations)
  T* s_zr = s_tile + S::NBUF * S::TILE;         // 2 x ZR
  T* s_yr = s_zr + 2 * S::ZR;                   // 2 x YR
  T* s_bt = s_yr + 2 * S::YR;                   // BT: staged z and y band rows (boundary tiles)
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int Nx = prm.Nx, Ny = prm.Ny, Nz = prm.Nz, pitch = prm.pitch;
  const long long sxy = (long long)pitch * Ny;
  // tile-level interior tests (band rows of all outputs of the tile)
  const bool inZ = z0 >= prm.st[2].lo && z0 + TZ - 1 <= prm.st[2].hi;
  const bool inY = y0 >= prm.st[1].lo && y0 + TY - 1 <= prm.st[1].hi;
  // x pass: two consecutive x (xp) in the (z',y) rows rg, rg + RG, ...
  const int xp = (tid % 16) * 2, rg = tid / 16;
  const bool inX = x0 + xp >= prm.st[0].lo && x0 + xp + 1 <= prm.st[0].hi;
  T cf[3][RPT][2], acc[3][RPT][2];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = r * RG + rg, zz = row / TY, yy = row % TY;
    const int gz = z0 + zz, gy = y0 + yy;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gx = x0 + xp + j;
      const bool in = gx < Nx && gy < Ny && gz < Nz;
      const long long g = gz * sxy + (long long)gy * pitch + gx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cf[c][r][j] = in ? prm.coef[1 + c][g] : T(0);
        acc[c][r][j] = T(0);
      }
    }
  }
  if (!inZ || !inY) {  // band rows of the tile's output rows (clamped to the last row), ops M, A, B
    constexpr int W = 2 * P + 1;
    for (int i = tid; i < S::BT; i += NT) {
      const int q = i % S::WP, r = (i / S::WP) % (TZ + TY), o = i / (S::WP * (TZ + TY));
      const bool isz = r < TZ;  // z rows first, then y rows ([op][row] per axis)
      const int d = isz ? 2 : 1, row = isz ? z0 + r : y0 + (r - TZ), Nd = isz ? Nz : Ny;
      const T* b = o == 0 ? prm.ax[d].band[OP_M] : (o == 1 ? prm.ax[d].band[OP_A] : prm.ax[d].band[OP_B]);
      const int dst = isz ? (o * TZ + r) * S::WP + q : 3 * TZ * S::WP + (o * TY + (r - TZ)) * S::WP + q;
      s_bt[dst] = q < W ? b[min(row, Nd - 1) * W + q] : T(0);
    }
  }
  if (tid == 0) {
    mbar_init(&bars[0]);
    mbar_init(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) tma_tile<T, P>(&maps.m[0], s_tile, &bars[0], x0 - 4, y0 - P, z0 - P);
  bool ok = pipe_field<T, P, H, 0>(prm, maps, s_tile, s_zr, s_yr, s_bt, bars, x0, y0, z0, inZ, inY, inX, xp, rg, cf, acc);
  if (ok) ok = pipe_field<T, P, H, 1>(prm, maps, s_tile, s_zr, s_yr, s_bt, bars, x0, y0, z0, inZ, inY, inX, xp, rg, cf, acc);
  if (ok) ok = pipe_field<T, P, H, 2>(prm, maps, s_tile, s_zr, s_yr, s_bt, bars, x0, y0, z0, inZ, inY, inX, xp, rg, cf, acc);
  if (ok) ok = pipe_field<T, P, H, 3>(prm, maps, s_tile, s_zr, s_yr, s_bt, bars, x0, y0, z0, inZ, inY, inX, xp, rg, cf, acc);
  if (ok) ok = pipe_field<T, P, H, 4>(prm, maps, s_tile, s_zr, s_yr, s_bt, bars, x0, y0, z0, inZ, inY, inX, xp, rg, cf, acc);
  if (ok) ok = pipe_field<T, P, H, 5>(prm, maps, s_tile, s_zr, s_yr, s_bt, bars, x0, y0, z0, inZ, inY, inX, xp, rg, cf, acc);
  if (ok) xstage<T, P, H, 5>(prm, s_yr, x0, inX, xp, rg, cf, acc);
  if (!ok) {
    // a tile never arrived: report, give the copies in flight a bounded time, leave
    if (tid == 0) atomicOr(prm.err, 1);
    mbar_wait(&bars[0], 0);
    mbar_wait(&bars[1], 0);
    return;
  }

  // ---- point source (only tiles holding its support evaluate g) and store
  double g = 0.0;
  if (prm.src_comp >= 0 && src_in_tile(prm.src_i0, P, x0, y0, z0, TX, TY, TZ)) {
    double tm = *prm.clock_t0 + ((double)*prm.clock_step + prm.t_frac) * prm.tau;
    double u = tm - prm.src_t0;
    g = prm.src_amp * sin(2.0 * 3.14159265358979323846 * prm.src_f0 * u) * exp(-(u / prm.src_s) * (u / prm.src_s));
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int row = r * RG + rg, zz = row / TY, yy = row % TY;
      const int gz = z0 + zz, gy = y0 + yy;
      if (gz >= Nz || gy >= Ny) continue;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int gx = x0 + xp + j;
        if (gx >= Nx) continue;
        T v = acc[c][r][j];
        if (c == prm.src_comp) {
          int ix = gx - prm.src_i0[0], iy = gy - prm.src_i0[1], iz = gz - prm.src_i0[2];
          if (ix >= 0 && ix <= P && iy >= 0 && iy <= P && iz >= 0 && iz <= P)
            v -= cf[1][r][j] * T(g) * prm.src_w[0][ix] * prm.src_w[1][iy] * prm.src_w[2][iz];
        }
        prm.out[c][gz * sxy + (long long)gy * pitch + gx] = v;
      }
    }
  }
}

// ------------------------------------------------- bounded-wait self-test
// Runs one of the kernels' bounded waits (which = 0: the E right-hand side's
// tile wait, 1: the x line solves' bulk-copy wait) on a barrier that expects
// bytes no copy will ever deliver: nothing is issued, so nothing is in flight
// when the wait gives up.  On give-up the kernel records it in the device status
// word exactly as the step kernels do (bit 0), which the host reports as
// ADI_ETIMEOUT.
__global__ void wait_selftest_kernel(int which, int budget, int* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  rhs2::mbar_init(&bar);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  xw_bar_expect(&bar, 16);  // one arrival, 16 bytes that never come
  const bool ok = which == 0 ? rhs2::mbar_wait(&bar, 0, budget) : xw_bar_wait(&bar, 0, budget);
  if (!ok) atomicOr(err, 1);
}

// ------------------------------------------------------------ conversions
__device__ __forceinline__ bool constrained(int comp, int i, int j, int k, int Nx, int Ny, int Nz) {
  // E_i (comp 0..2): zero ends in the two directions != i; H_i: in direction i
  bool bx = (i == 0 || i == Nx - 1), by = (j == 0 || j == Ny - 1), bz = (k == 0 || k == Nz - 1);
  switch (comp) {
    case 0: return by || bz;
    case 1: return bx || bz;
    case 2: return bx || by;
    case 3: return bx;
    case 4: return by;
    default: return bz;
  }
}

// Flat element g of the dense host layout (component, then z, y, x) and its
// successor.
__device__ __forceinline__ void flat_pos(long long g, long long Nc, int Nx, int Ny, int& comp, int& i, int& j, int& k) {
  comp = (int)(g / Nc);
  const long long r = g - comp * Nc, jk = r / Nx;
  i = (int)(r - jk * Nx);
  k = (int)(jk / Ny);
  j = (int)(jk - (long long)k * Ny);
}
__device__ __forceinline__ void flat_next(int& comp, int& i, int& j, int& k, int Nx, int Ny, int Nz) {
  if (++i == Nx) {
    i = 0;
    if (++j == Ny) {
      j = 0;
      if (++k == Nz) {
        k = 0;
        ++comp;
      }
    }
  }
}

// V consecutive elements of type S as one 16-byte access (V = 1: scalar)
template <typename S, int V>
struct Vec;
template <typename S>
struct Vec<S, 1> {
  static __device__ __forceinline__ void ld(const S* p, S (&e)[1]) { e[0] = p[0]; }
  static __device__ __forceinline__ void st(S* p, const S (&e)[1]) { p[0] = e[0]; }
};
template <>
struct Vec<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&e)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    e[0] = v.x, e[1] = v.y, e[2] = v.z, e[3] = v.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&e)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(e[0], e[1], e[2], e[3]);
  }
};
template <>
struct Vec<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&e)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    e[0] = v.x, e[1] = v.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&e)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(e[0], e[1]);
  }
};

// Dense host layout (src, element type S; may be host memory mapped into the
// device address space, read V elements per access) -> the pitched state
// (element type T), zeroing the coefficients fixed by the boundary conditions;
// bad (optional) receives 1 if any source value is NaN or Inf.
template <typename S, typename T, int V>
__global__ void set_fields_kernel(const S* __restrict__ src, T* d0, T* d1, T* d2, T* d3, T* d4, T* d5, int Nx, int Ny,
                                  int Nz, int pitch, int* bad) {
  const long long Nc = (long long)Nx * Ny * Nz, n = 6 * Nc, nv = n / V;
  T* dst[6] = {d0, d1, d2, d3, d4, d5};
  int local_bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv + (n - nv * V); v += stride) {
    // vectors first, then the (fewer than V) remaining elements one by one
    const bool vec = v < nv;
    const long long g = vec ? v * V : nv * V + (v - nv);
    int comp, i, j, k;
    flat_pos(g, Nc, Nx, Ny, comp, i, j, k);
    S e[V];
    if (vec) {
      Vec<S, V>::ld(src + g, e);
    } else {
      e[0] = src[g];
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
      if (!vec && u > 0) break;
      if (!isfinite(e[u])) local_bad = 1;
      dst[comp][((long long)k * Ny + j) * pitch + i] = constrained(comp, i, j, k, Nx, Ny, Nz) ? T(0) : T(e[u]);
      flat_next(comp, i, j, k, Nx, Ny, Nz);
    }
  }
  if (bad && __syncthreads_or(local_bad) && threadIdx.x == 0) atomicOr(bad, 1);
}

template <typename S>
__global__ void finite_kernel(const S* __restrict__ src, long long n, int* bad) {
  int local_bad = 0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x)
    if (!isfinite(src[g])) local_bad = 1;
  if (__syncthreads_or(local_bad) && threadIdx.x == 0) atomicOr(bad, 1);
}

// The pitched state (T) -> the dense layout (S, possibly mapped host memory,
// written V elements per access); bad receives 1 if any value is NaN or Inf.
template <typename S, typename T, int V>
__global__ void get_fields_kernel(S* __restrict__ dst, const T* s0, const T* s1, const T* s2, const T* s3,
                                  const T* s4, const T* s5, int Nx, int Ny, int Nz, int pitch, int* bad) {
  const T* src[6] = {s0, s1, s2, s3, s4, s5};
  const long long Nc = (long long)Nx * Ny * Nz, n = 6 * Nc, nv = n / V;
  int local_bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv + (n - nv * V); v += stride) {
    const bool vec = v < nv;
    const long long g = vec ? v * V : nv * V + (v - nv);
    int comp, i, j, k;
    flat_pos(g, Nc, Nx, Ny, comp, i, j, k);
    S e[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      if (!vec && u > 0) break;
      e[u] = (S)src[comp][((long long)k * Ny + j) * pitch + i];
      if (!isfinite(e[u])) local_bad = 1;
      flat_next(comp, i, j, k, Nx, Ny, Nz);
    }
    if (vec) Vec<S, V>::st(dst + g, e);
    else dst[g] = e[0];
  }
  if (local_bad) atomicOr(bad, 1);
}

// The state's six arrays from the six scratch arrays (16-byte words, n per
// array) and the clock, only if the conversion into scratch found every value
// finite; otherwise the refusal is recorded and nothing changes.
struct CommitArgs {
  const uint4* src[6];
  uint4* dst[6];
};
__global__ void commit_kernel(const CommitArgs a, long long n, const int* bad, int* refused, double* t0,
                              long long* step, double t) {
  if (*bad) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(refused, 1);
    return;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 6 * n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / n);
    const long long j = i - c * n;
    a.dst[c][j] = a.src[c][j];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *t0 = t;
    *step = 0;
  }
}

__global__ void clock_kernel(double* t0, long long* step, double t) {
  *t0 = t;
  *step = 0;
}

__global__ void clock_advance_kernel(long long* step) { *step += 1; }

// Per-row material (support-weighted mean of per-element data) and the row
// coefficients a, b, c, d; also the running minimum of eps^ mu^.
template <typename T>
__global__ void coef_kernel(const double* __restrict__ eps, const double* __restrict__ mu,
                            const double* __restrict__ sig, const double* __restrict__ Gx,
                            const double* __restrict__ Gy, const double* __restrict__ Gz, int nx, int ny,
                            int nz, int p, int pitch, double tau, T* ca, T* cb, T* cc, T* cd,
                            unsigned long long* min_bits) {
  const int Nx = nx + p, Ny = ny + p, Nz = nz + p;
  const long long Nc = (long long)Nx * Ny * Nz;
  double local_min = 1e300;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < Nc;
       g += (long long)gridDim.x * blockDim.x) {
    int r = (int)(g % Nx), s = (int)((g / Nx) % Ny), t = (int)(g / ((long long)Nx * Ny));
    double ne = 0, nm = 0, ns = 0, den = 0;
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
          ne += w * eps[e];
          nm += w * mu[e];
          ns += w * sig[e];
          den += w;
        }
      }
    }
    double eh = ne / den, mh = nm / den, sh = ns / den;
    double alpha = sh * tau / (4.0 * eh);
    const long long o = ((long long)t * Ny + s) * pitch + r;
    ca[o] = T((1.0 - alpha) / (1.0 + alpha));
    cb[o] = T(tau / (2.0 * eh * (1.0 + alpha)));
    cc[o] = T(tau * tau / (4.0 * eh * mh * (1.0 + alpha)));
    cd[o] = T(tau / (2.0 * mh));
    local_min = fmin(local_min, eh * mh);
  }
  // positive doubles order like their bit patterns
  atomicMin(min_bits, (unsigned long long)__double_as_longlong(local_min));
}

// ---------------------------------------------------------------- helpers
template <typename T>
struct Layout {
  // offsets (elements of T) of the 1D tables of axis d inside c.tab
  size_t band[3][4];
  size_t lu[3][2][3];
  size_t total;
};

template <typename T>
Layout<T> table_layout(const Ctx& c) {
  Layout<T> L{};
  size_t off = 0;
  const int p = c.p, W = 2 * p + 1;
  for (int d = 0; d < 3; ++d) {
    int N = c.N[d];
    for (int o = 0; o < 4; ++o) {
      L.band[d][o] = off;
      off += (size_t)N * W;
    }
    for (int f = 0; f < 2; ++f) {
      L.lu[d][f][0] = off;
      off += (size_t)N * p;
      L.lu[d][f][1] = off;
      off += (size_t)N;
      L.lu[d][f][2] = off;
      off += (size_t)N * p;
    }
  }
  L.total = off;
  return L;
}

template <typename T>
AxisDev<T> axis_dev(const Ctx& c, int d) {
  Layout<T> L = table_layout<T>(c);
  const T* base = reinterpret_cast<const T*>(c.tab);
  AxisDev<T> a;
  for (int o = 0; o < 4; ++o) a.band[o] = base + L.band[d][o];
  for (int f = 0; f < 2; ++f) {
    a.luL[f] = base + L.lu[d][f][0];
    a.luInv[f] = base + L.lu[d][f][1];
    a.luU[f] = base + L.lu[d][f][2];
  }
  a.N = c.N[d];
  const Axis1D& h = c.axes[d];
  const int p = h.p, W = 2 * p + 1;
  a.inner_lo = h.inner_lo;  // the rows with the interior stencil (detected by build_axis)
  a.inner_hi = h.inner_hi;
  for (int o = 0; o < 4; ++o)
    for (int q = 0; q < 2 * kMaxP + 1; ++q) a.inner[o][q] = T(0);
  if (a.inner_lo <= a.inner_hi) {
    const std::vector<double>* src[4] = {&h.M, &h.S, &h.A, &h.B};
    for (int o = 0; o < 4; ++o)
      for (int q = 0; q < W; ++q) a.inner[o][q] = T((*src[o])[(size_t)a.inner_lo * W + q]);
  }
  for (int f = 0; f < 2; ++f) {
    const LuConst& lc = c.luconst[d][f];
    a.lu_lo[f] = lc.lo;
    a.lu_hi[f] = lc.hi;
    for (int q = 0; q < 3 * kMaxP + 1; ++q) a.luc[f][q] = T(q < 3 * p + 1 ? lc.v[q] : 0.0);
  }
  return a;
}

// element blocks of the 1D matrices (rhs_quad), per axis, in the working precision
template <typename T>
cudaError_t upload_quad_tables(Ctx& c) {
  std::vector<T> h;
  for (int d = 0; d < 3; ++d) {
    std::vector<double> loc;
    element_matrices(c.axes[d], loc);
    for (double v : loc) h.push_back(T(v));
  }
  if (!c.tabq) {
    cudaError_t e = cudaMalloc(&c.tabq, h.size() * sizeof(T));
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpyAsync(c.tabq, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  return e;
}

template <typename T>
cudaError_t upload_tables_t(Ctx& c) {
  Layout<T> L = table_layout<T>(c);
  std::vector<T> h(L.total, T(0));
  const int p = c.p;
  for (int d = 0; d < 3; ++d) {
    const Axis1D& ax = c.axes[d];
    const std::vector<double>* src[4] = {&ax.M, &ax.S, &ax.A, &ax.B};
    for (int o = 0; o < 4; ++o)
      for (size_t i = 0; i < src[o]->size(); ++i) h[L.band[d][o] + i] = T((*src[o])[i]);
    for (int f = 0; f < 2; ++f) {
      BandLU lu;
      int N = ax.N;
      band_lu(ax.M, nullptr, N, p, f ? 1 : 0, f ? N - 2 : N - 1, lu);
      // rows whose factors round to the mid-line factors in T
      {
        auto vals = [&](int r, double* v) {
          for (int q = 0; q < p; ++q) {
            v[q] = lu.L[(size_t)r * p + q];
            v[p + 1 + q] = lu.U[(size_t)r * p + q];
          }
          v[p] = lu.inv_d[r];
        };
        auto same = [&](int r, const double* ref) {
          double v[3 * kMaxP + 1];
          vals(r, v);
          for (int q = 0; q < 3 * p + 1; ++q)
            if (T(v[q]) != T(ref[q])) return false;
          return true;
        };
        LuConst& lc = c.luconst[d][f];
        const int mid = N / 2;
        vals(mid, lc.v);
        lc.lo = mid;
        while (lc.lo - 1 >= (f ? 1 : 0) && same(lc.lo - 1, lc.v)) --lc.lo;
        lc.hi = mid;
        while (lc.hi + 1 <= (f ? N - 2 : N - 1) && same(lc.hi + 1, lc.v)) ++lc.hi;
        if (N < 8) {
          lc.lo = 1;
          lc.hi = 0;
        }
      }
      for (int k = 0; k < N; ++k) {
        h[L.lu[d][f][1] + k] = T(lu.inv_d[k]);
        for (int q = 0; q < p; ++q) {
          h[L.lu[d][f][0] + (size_t)k * p + q] = T(lu.L[(size_t)k * p + q]);
          h[L.lu[d][f][2] + (size_t)k * p + q] = T(lu.U[(size_t)k * p + q]);
        }
      }
    }
  }
  if (c.tab && c.tab_bytes != L.total * sizeof(T)) {
    cudaFree(c.tab);
    c.tab = nullptr;
  }
  if (!c.tab) {
    cudaError_t e = cudaMalloc(&c.tab, L.total * sizeof(T));
    if (e != cudaSuccess) return e;
    c.tab_bytes = L.total * sizeof(T);
  }
  cudaError_t e = cudaMemcpyAsync(c.tab, h.data(), L.total * sizeof(T), cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c.stream);
}

// Terms of the E right-hand side (eq. dupa1ab and its half step 2 analogue).
// fields: 0..2 = E1..E3, 3..5 = H1..H3 (old level).
int e_terms(int half, Term* t) {
  auto T_ = [](int f, int out, int ox, int oy, int oz, int cf, float s) {
    Term x;
    x.field = f;
    x.out = out;
    x.op[0] = ox;
    x.op[1] = oy;
    x.op[2] = oz;
    x.coef = cf;
    x.sign = s;
    return x;
  };
  int n = 0;
  // E fields: a M(x)M(x)M E_i, and the R cross terms scaled by c
  if (half == 1) {
    t[n++] = T_(0, 0, OP_M, OP_M, OP_M, CF_A, 1.f);
    t[n++] = T_(0, 2, OP_B, OP_M, OP_A, CF_C, 1.f);  // R1[3][1] = B(x)M(x)A
    t[n++] = T_(1, 1, OP_M, OP_M, OP_M, CF_A, 1.f);
    t[n++] = T_(1, 0, OP_A, OP_B, OP_M, CF_C, 1.f);  // R1[1][2] = A(x)B(x)M
    t[n++] = T_(2, 2, OP_M, OP_M, OP_M, CF_A, 1.f);
    t[n++] = T_(2, 1, OP_M, OP_A, OP_B, CF_C, 1.f);  // R1[2][3] = M(x)A(x)B
  } else {
    t[n++] = T_(0, 0, OP_M, OP_M, OP_M, CF_A, 1.f);
    t[n++] = T_(0, 1, OP_B, OP_A, OP_M, CF_C, 1.f);  // R2[2][1] = B(x)A(x)M
    t[n++] = T_(1, 1, OP_M, OP_M, OP_M, CF_A, 1.f);
    t[n++] = T_(1, 2, OP_M, OP_B, OP_A, CF_C, 1.f);  // R2[3][2] = M(x)B(x)A
    t[n++] = T_(2, 2, OP_M, OP_M, OP_M, CF_A, 1.f);
    t[n++] = T_(2, 0, OP_A, OP_M, OP_B, CF_C, 1.f);  // R2[1][3] = A(x)M(x)B
  }
  // curl H = (C1 - C2) H, scaled by b
  t[n++] = T_(3, 1, OP_M, OP_M, OP_A, CF_B, 1.f);   // + d3 H1 -> E2
  t[n++] = T_(3, 2, OP_M, OP_A, OP_M, CF_B, -1.f);  // - d2 H1 -> E3
  t[n++] = T_(4, 0, OP_M, OP_M, OP_A, CF_B, -1.f);  // - d3 H2 -> E1
  t[n++] = T_(4, 2, OP_A, OP_M, OP_M, CF_B, 1.f);   // + d1 H2 -> E3
  t[n++] = T_(5, 0, OP_M, OP_A, OP_M, CF_B, 1.f);   // + d2 H3 -> E1
  t[n++] = T_(5, 1, OP_A, OP_M, OP_M, CF_B, -1.f);  // - d1 H3 -> E2
  return n;
}

// Terms of the H right-hand side: M H_old - d C1 E_alpha + d C2 E_beta.
// fields: 0..2 = H_old, 3..5 = E_alpha, 6..8 = E_beta.
int h_terms(Term* t) {
  auto T_ = [](int f, int out, int ox, int oy, int oz, int cf, float s) {
    Term x;
    x.field = f;
    x.out = out;
    x.op[0] = ox;
    x.op[1] = oy;
    x.op[2] = oz;
    x.coef = cf;
    x.sign = s;
    return x;
  };
  int n = 0;
  t[n++] = T_(0, 0, OP_M, OP_M, OP_M, CF_ONE, 1.f);
  t[n++] = T_(1, 1, OP_M, OP_M, OP_M, CF_ONE, 1.f);
  t[n++] = T_(2, 2, OP_M, OP_M, OP_M, CF_ONE, 1.f);
  t[n++] = T_(3, 1, OP_M, OP_M, OP_A, CF_D, -1.f);  // (C1 E)2 = d3 E1
  t[n++] = T_(4, 2, OP_A, OP_M, OP_M, CF_D, -1.f);  // (C1 E)3 = d1 E2
  t[n++] = T_(5, 0, OP_M, OP_A, OP_M, CF_D, -1.f);  // (C1 E)1 = d2 E3
  t[n++] = T_(6, 2, OP_M, OP_A, OP_M, CF_D, 1.f);   // (C2 E)3 = d2 E1
  t[n++] = T_(7, 0, OP_M, OP_M, OP_A, CF_D, 1.f);   // (C2 E)1 = d3 E2
  t[n++] = T_(8, 1, OP_A, OP_M, OP_M, CF_D, 1.f);   // (C2 E)2 = d1 E3
  return n;
}

template <typename T, int P>
constexpr int rhs_tz() { return 8; }

template <typename T, int P>
size_t rhs_smem() {
  constexpr int TX = 32, TY = 8, TZ = 8;
  return sizeof(T) * ((size_t)(TZ + 2 * P) * (TY + 2 * P) * (TX + 2 * P) + (size_t)TZ * (TY + 2 * P) * (TX + 2 * P) +
                      (size_t)TZ * TY * (TX + 2 * P));
}

template <int P>
size_t resid_ff_smem() {
  constexpr int TX = 32, TY = 8, TZ = 8;
  const size_t nin = (size_t)(TZ + 2 * P) * (TY + 2 * P) * (TX + 2 * P);
  return sizeof(float) * ((nin + 1) & ~(size_t)1) +
         sizeof(float) * 2 * ((size_t)TZ * (TY + 2 * P) * (TX + 2 * P) + (size_t)TZ * TY * (TX + 2 * P));
}

template <typename T, int P>
cudaError_t launch_rhs(Ctx& c, RhsParams<T>& prm, const char* name, double bytes) {
  constexpr int TX = 32, TY = 8, TZ = 8;
  size_t smem = rhs_smem<T, P>();
  auto kern = rhs_kernel<T, P, TX, TY, TZ>;
  dim3 grid((c.N[0] + TX - 1) / TX, (c.N[1] + TY - 1) / TY, (c.N[2] + TZ - 1) / TZ);
  prof_begin(c, name, bytes);
  kern<<<grid, dim3(TX, TY), smem, c.stream>>>(prm);
  prof_end(c);
  return cudaGetLastError();
}

cudaError_t advance_clock(Ctx& c) {
  prof_begin(c, "clock", 0.0);
  clock_advance_kernel<<<1, 1, 0, c.stream>>>(c.d_clock_step);
  prof_end(c);
  return cudaGetLastError();
}

template <typename T, int P>
size_t rhs_e_smem() {
  return rhs2::Smem<T, P>::BYTES;
}

// TMA descriptor of one state array: dims (N_x, N_y, N_z), row pitch c.pitch,
// box (40, 8 + 2p, 8 + 2p) for the E right-hand side tiles.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_map(Ctx& c, EncodeTiledFn fn, void* base, CUtensorMap* out) {
  const cuuint64_t dims[3] = {(cuuint64_t)c.N[0], (cuuint64_t)c.N[1], (cuuint64_t)c.N[2]};
  const cuuint64_t strides[2] = {(cuuint64_t)c.pitch * c.esize, (cuuint64_t)c.pitch * c.N[1] * c.esize};
  const cuuint32_t box[3] = {(cuuint32_t)rhs2::BOXX, (cuuint32_t)(rhs2::TY + 2 * c.p), (cuuint32_t)(rhs2::TZ + 2 * c.p)};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(out, c.precision == ADI_PREC_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T>
Stencils<T> stencils_of(const Axis1D& ax) {
  Stencils<T> s{};
  const int p = ax.p, W = 2 * p + 1;
  s.lo = ax.inner_lo;  // the rows with the interior stencil (detected by build_axis)
  s.hi = ax.inner_hi;
  if (s.lo <= s.hi) {
    const std::vector<double>* src[3] = {&ax.M, &ax.A, &ax.B};
    for (int o = 0; o < 3; ++o)
      for (int q = 0; q < W; ++q) s.w[o][q] = T((*src[o])[(size_t)s.lo * W + q]);
  }
  return s;
}

template <typename T, int P>
cudaError_t launch_rhs_e(Ctx& c, RhsParams<T>& prm, int half, double bytes, bool bf16_tiles) {
  using namespace rhs2;
  if (!c.tmaps_ok) return cudaErrorInvalidValue;
  for (int d = 0; d < 3; ++d) prm.st[d] = stencils_of<T>(c.axes[d]);
  prm.err = c.d_err;
  TmaMaps maps;
  for (int i = 0; i < 3; ++i) {
    maps.m[i] = half == 1 ? c.tmap_cur[i] : c.tmap_half[i];  // E^n or E^{n+1/2}
    maps.m[3 + i] = c.tmap_cur[3 + i];                         // H (one buffer)
  }
  dim3 grid((c.N[0] + TX - 1) / TX, (c.N[1] + TY - 1) / TY, (c.N[2] + TZ - 1) / TZ);
  bool done = false;
  if constexpr (sizeof(T) == 4) {  // mixed mode: BF16 operands on the tensor cores (the generic term list)
    if (bf16_tiles) {
      prof_begin(c, "rhs_E_mma", bytes);
      rhs_e_mma_kernel<P><<<grid, dim3(32, 8), MmaTile<P>::BYTES, c.stream>>>(prm);
      done = true;
    }
  }
  if (!done) prof_begin(c, "rhs_E", bytes);
  if (!done) {
    if (half == 1) rhs_e_kernel<T, P, 1><<<grid, NT, rhs_e_smem<T, P>(), c.stream>>>(prm, maps);
    else rhs_e_kernel<T, P, 2><<<grid, NT, rhs_e_smem<T, P>(), c.stream>>>(prm, maps);
  }
  prof_end(c);
  return cudaGetLastError();
}

template <typename T, int P>
cudaError_t launch_line(Ctx& c, int dir, int mode, const LineJobs<T>& jobs, int njobs, const char* name) {
  LineParams lp;
  lp.dir = dir;
  lp.N = c.N[dir];
  lp.Nx = c.N[0];
  lp.Ny = c.N[1];
  lp.Nz = c.N[2];
  lp.pitch = c.pitch;
  lp.err = c.d_err;
  lp.nlines = (long long)c.N[0] * c.N[1] * c.N[2] / c.N[dir];
  const double per_job = (double)c.Nc * sizeof(T) *
                         (mode == LM_MASS || mode == LM_PIVOT ? 2.0 : (mode == LM_STIFF ? 4.0 : 3.0));
  // y and z stiffness lines: the streaming kernel with precomputed factors (no
  // shared memory).  Mass and derivative lines stay on the staged kernel: their
  // streaming forms measured slower (the forward sweep's intermediate of a whole
  // launch, 1 KB per line, does not stay in L2 for the backward sweep).
  const bool stream_ok = dir != 0 && mode == LM_STIFF && jobs.job[0].fac[0] != nullptr && c.line_stream;
  if (stream_ok) {
    const AxisDev<T> axs = axis_dev<T>(c, dir);
    dim3 g2((unsigned)((lp.nlines + 127) / 128), njobs);
    prof_begin(c, name, per_job * njobs);
    if (mode == LM_STIFF) line_direct_kernel<T, P, LM_STIFF><<<g2, 128, 0, c.stream>>>(jobs, lp, axs);
    else if (mode == LM_DERIV) line_direct_kernel<T, P, LM_DERIV><<<g2, 128, 0, c.stream>>>(jobs, lp, axs);
    else line_direct_kernel<T, P, LM_MASS><<<g2, 128, 0, c.stream>>>(jobs, lp, axs);
    prof_end(c);
    return cudaGetLastError();
  }
  // x lines on one warp per 32 lines: rows [line][k] of shared memory with a pitch lpk of a
  // multiple of 4 elements, lpk / 4 odd (conflict-free 16-byte lane accesses in FP32)
  // a line padded to 4 elements, plus 12 elements of slack (the derivative sweep
  // reads up to 4 (NV - 1) <= 8 rows beyond its block of 4, plus one block ahead)
  int lpk = ((lp.N + 3) & ~3) + 12;
  if (((lpk >> 2) & 1) == 0) lpk += 4;
  const size_t smw = sizeof(T) * 32 * (size_t)lpk;
  // x stiffness lines with precomputed row factors (FP32 and FP64): plane plus a two-stage ring
  const size_t sms = smw + sizeof(T) * 2 * (P + 1) * 32 * (xws_rows<T>() + 4);
  bool xs = dir == 0 && mode == LM_STIFF && c.line_xw && jobs.job[0].fac[0] != nullptr;
  for (int j = 0; j < njobs && xs; ++j) {  // 16-byte aligned line starts (pitch is a multiple of 4)
    uintptr_t a = reinterpret_cast<uintptr_t>(jobs.job[j].src) | reinterpret_cast<uintptr_t>(jobs.job[j].dst) |
                  reinterpret_cast<uintptr_t>(jobs.job[j].aux2);
    for (int m = 0; m < 2 * P; ++m) a |= reinterpret_cast<uintptr_t>(jobs.job[j].fac[m]);
    xs = (a & 15) == 0 && jobs.job[j].aux2 != nullptr;
  }
  if (xs && sms <= (size_t)c.smem_optin) {
    dim3 gs((unsigned)((lp.nlines + 31) / 32), njobs);
    prof_begin(c, name, per_job * njobs);
    line_xws_kernel<T, P><<<gs, 32, sms, c.stream>>>(jobs, lp, lpk);
    prof_end(c);
    return cudaGetLastError();
  }
  if constexpr (sizeof(T) == 4) {
    // x mass and derivative lines (FP32): whole-line bulk copies
    bool xw = dir == 0 && (mode == LM_MASS || mode == LM_DERIV) && c.line_xw;
    for (int j = 0; j < njobs; ++j)
      xw = xw && ((reinterpret_cast<uintptr_t>(jobs.job[j].src) | reinterpret_cast<uintptr_t>(jobs.job[j].dst)) & 15) == 0;
    if (xw && smw <= (size_t)c.smem_optin) {
      const AxisDev<T> axw = axis_dev<T>(c, 0);
      dim3 gw((unsigned)((lp.nlines + 31) / 32), njobs);
      prof_begin(c, name, per_job * njobs);
      if (mode == LM_MASS) line_xw_kernel<P, LM_MASS><<<gw, 32, smw, c.stream>>>(jobs, lp, axw, lpk);
      else line_xw_kernel<P, LM_DERIV><<<gw, 32, smw, c.stream>>>(jobs, lp, axw, lpk);
      prof_end(c);
      return cudaGetLastError();
    }
  }
  const int W = 2 * P + 1;
  const bool fact = mode == LM_STIFF || mode == LM_PIVOT;
  const int tabw = fact ? 2 * W : (mode == LM_DERIV ? 3 * P + 1 + W : 3 * P + 1);
  // shared planes: rhs/result, then c, pivots and the P upper-factor planes
  const int planes = mode == LM_STIFF ? 1 + (P > 2 ? P : 2) : (mode == LM_PIVOT ? 2 : 1);
  const size_t limit = (size_t)c.smem_optin;
  auto smem_for = [&](int lines) {
    const int lp_ = dir == 0 ? lines + 1 : lines;
    return sizeof(T) * ((((size_t)lp.N * tabw + 3) & ~(size_t)3) + (size_t)planes * lp.N * lp_);
  };
  // largest tile (<= 64 lines) that leaves room for two CTAs per SM
  int lines = 64;
  while (lines > 8 && smem_for(lines) > limit / 2) lines /= 2;
  if (c.line_tile > 0 && smem_for(c.line_tile) <= limit) lines = c.line_tile;  // autotuned width
  if (smem_for(lines) > limit) return cudaErrorInvalidValue;
  size_t smem = smem_for(lines);
  long long blocks = (lp.nlines + lines - 1) / lines;
  prof_begin(c, name, per_job * njobs);
  dim3 grid((unsigned)blocks, njobs);
  const AxisDev<T> ax = axis_dev<T>(c, dir);
  const bool x = dir == 0;
  if (mode == LM_STIFF) {
    if (x) line_kernel<T, P, LM_STIFF, true><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
    else line_kernel<T, P, LM_STIFF, false><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
  } else if (mode == LM_PIVOT) {
    if (x) line_kernel<T, P, LM_PIVOT, true><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
    else line_kernel<T, P, LM_PIVOT, false><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
  } else if (mode == LM_DERIV) {
    if (x) line_kernel<T, P, LM_DERIV, true><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
    else line_kernel<T, P, LM_DERIV, false><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
  } else {
    if (x) line_kernel<T, P, LM_MASS, true><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
    else line_kernel<T, P, LM_MASS, false><<<grid, lines, smem, c.stream>>>(jobs, lp, ax);
  }
  prof_end(c);
  return cudaGetLastError();
}

template <typename T>
LineJob<T> job_of(const T* src, T* dst, const T* aux, double scale, int dirichlet, const T* aux2 = nullptr) {
  LineJob<T> j;
  j.src = src;
  j.dst = dst;
  j.aux = aux;
  j.aux2 = aux2;
  j.scale = T(scale);
  j.dirichlet = dirichlet;
  j.work = nullptr;
  for (int m = 0; m < 2 * kMaxP; ++m) j.fac[m] = nullptr;
  return j;
}

// stiffness direction of E_i: half 1 (y, z, x), half 2 (z, x, y)
constexpr int kStiffDir[2][3] = {{1, 2, 0}, {2, 0, 1}};

// Solve T E = R per component: the stiffness direction first, then the two
// mass directions (order of the Appendix, eqs. split1/split2); R is overwritten
// and the result goes to out (may be R itself).
// The three components of an E half step (and the three H components of the
// uniform-mu H half step) are independent chains of line solves that write
// disjoint arrays.  Chains runs chain i on branch stream i, forked from and
// joined back to c.stream; inside a captured step they become parallel branches
// of the graph, so the short, latency-bound line solves of different
// components share the SMs.  Each chain keeps its own order, hence the same
// results bit for bit as the serial order.  While profiling (per-launch events
// on c.stream) and with serial_chains the chains run one after another.
class Chains {
 public:
  explicit Chains(Ctx& c) : c_(c), main_(c.stream), on_(!c.profiling && !c.serial_chains && c.branch[0]) {
    if (!on_) return;
    err_ = cudaEventRecord(c.ev_fork, main_);
    for (int i = 0; i < 3 && err_ == cudaSuccess; ++i) err_ = cudaStreamWaitEvent(c.branch[i], c.ev_fork, 0);
  }
  ~Chains() { join(); }
  Chains(const Chains&) = delete;
  Chains& operator=(const Chains&) = delete;
  cudaError_t status() const { return err_; }
  void use(int i) {
    if (on_) c_.stream = c_.branch[i];
  }
  // main stream waits for every branch; c.stream is the main stream again
  cudaError_t join() {
    if (!on_) return cudaSuccess;
    on_ = false;
    c_.stream = main_;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
      e = cudaEventRecord(c_.ev_join[i], c_.branch[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(main_, c_.ev_join[i], 0);
    }
    return e;
  }

 private:
  Ctx& c_;
  cudaStream_t main_;
  bool on_;
  cudaError_t err_ = cudaSuccess;
};

// Line solves of E component i of half step `half`, in place on R[i] and into
// out[i]: the row-scaled M + c S along the material direction first (R10),
// then the two mass directions.
template <typename T, int P>
cudaError_t e_chain(Ctx& c, int half, int i, T* const* R, T* const* out) {
  T** cf = reinterpret_cast<T**>(c.coef);
  static const char* stiff_name[3] = {"line_x_stiff", "line_y_stiff", "line_z_stiff"};
  static const char* mass_name[3] = {"line_x_mass", "line_y_mass", "line_z_mass"};
  const int sd = kStiffDir[half - 1][i];
  LineJobs<T> js{};
  js.job[0] = job_of<T>(R[i], R[i], cf[2], 0.0, 1, reinterpret_cast<const T*>(c.pivots[sd]));
  for (int m = 0; m < 2 * P; ++m) js.job[0].fac[m] = reinterpret_cast<T*>(c.stiff_fac[sd][m]);
  cudaError_t e = launch_line<T, P>(c, sd, LM_STIFF, js, 1, stiff_name[sd]);
  if (e != cudaSuccess) return e;
  int md[2], m = 0;
  for (int d = 0; d < 3; ++d)
    if (d != sd) md[m++] = d;
  js.job[0] = job_of<T>(R[i], R[i], nullptr, 0.0, md[0] != i);
  e = launch_line<T, P>(c, md[0], LM_MASS, js, 1, mass_name[md[0]]);
  if (e != cudaSuccess) return e;
  js.job[0] = job_of<T>(R[i], out[i], nullptr, 0.0, md[1] != i);
  return launch_line<T, P>(c, md[1], LM_MASS, js, 1, mass_name[md[1]]);
}

template <typename T, int P>
cudaError_t e_solve(Ctx& c, int half, T* const* R, T* const* out) {
  Chains ch(c);
  cudaError_t e = ch.status();
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    ch.use(i);
    e = e_chain<T, P>(c, half, i, R, out);
  }
  const cudaError_t ej = ch.join();
  return e != cudaSuccess ? e : ej;
}

// FP64 band table of (axis d, op o) inside c.tab64
inline const double* band64(const Ctx& c, int d, int o) {
  size_t off = 0;
  const int W = 2 * c.p + 1;
  for (int k = 0; k < d; ++k) off += 4 * (size_t)c.N[k] * W;
  return c.tab64 + off + (size_t)o * c.N[d] * W;
}

template <int P>
cudaError_t launch_resid(Ctx& c, int half, float* const* Ein, float* const* Hin, float* const* Estar, float* const* R) {
  float** cf = reinterpret_cast<float**>(c.coef);
  ResidParams prm{};
  for (int i = 0; i < 3; ++i) {
    prm.fields[i] = Ein[i];
    prm.fields[3 + i] = Hin[3 + i];
    prm.fields[6 + i] = Estar[i];
    prm.out[i] = R[i];
  }
  prm.coef[CF_A] = cf[0];
  prm.coef[CF_B] = cf[1];
  prm.coef[CF_C] = cf[2];
  for (int d = 0; d < 3; ++d)
    for (int o = 0; o < 4; ++o) prm.band[d][o] = band64(c, d, o);
  int n = e_terms(half, prm.terms);
  for (int k = 0; k < 3; ++k) {
    Term t{};
    t.field = 6 + k;
    t.out = k;
    t.op[0] = t.op[1] = t.op[2] = OP_M;
    t.coef = CF_ONE;
    t.sign = -1.f;
    prm.terms[n++] = t;
    t.op[kStiffDir[half - 1][k]] = OP_S;
    t.coef = CF_C;
    prm.terms[n++] = t;
  }
  prm.nterms = n;
  prm.Nx = c.N[0];
  prm.Ny = c.N[1];
  prm.Nz = c.N[2];
  prm.pitch = c.pitch;
  prm.src_comp = (c.src_comp >= 0 && c.src_amp != 0.0) ? c.src_comp : -1;
  for (int d = 0; d < 3; ++d) {
    prm.src_i0[d] = c.src_i0[d];
    for (int q = 0; q <= kMaxP; ++q) prm.src_w[d][q] = c.src_w[d][q];
  }
  prm.src_amp = c.src_amp;
  prm.src_f0 = c.src_f0;
  prm.src_t0 = c.src_t0;
  prm.src_s = c.src_s;
  prm.tau = c.dt;
  prm.t_frac = half == 1 ? 0.25 : 0.75;
  prm.clock_t0 = c.d_clock_t0;
  prm.clock_step = c.d_clock_step;
  constexpr int TX = 32, TY = 8, TZ = 8;
  const size_t smem = sizeof(double) * ((size_t)(TZ + 2 * P) * (TY + 2 * P) * (TX + 2 * P) +
                                        (size_t)TZ * (TY + 2 * P) * (TX + 2 * P) + (size_t)TZ * TY * (TX + 2 * P));
  dim3 grid((c.N[0] + TX - 1) / TX, (c.N[1] + TY - 1) / TY, (c.N[2] + TZ - 1) / TZ);
  prof_begin(c, "resid_E64", (double)c.Nc * 4.0 * 15.0);  // reads 9 fields + a, b, c, writes 3
  resid_kernel<P><<<grid, dim3(TX, TY), smem, c.stream>>>(prm);
  prof_end(c);
  return cudaGetLastError();
}

// float-float band table of (axis d, op o) inside c.tabff
inline const float2* bandff(const Ctx& c, int d, int o) {
  size_t off = 0;
  const int W = 2 * c.p + 1;
  for (int k = 0; k < d; ++k) off += 4 * (size_t)c.N[k] * W;
  return c.tabff + off + (size_t)o * c.N[d] * W;
}

template <int P>
cudaError_t launch_resid_ff(Ctx& c, int half, float* const* Ein, float* const* Hin, float* const* Estar,
                            float* const* R) {
  float** cf = reinterpret_cast<float**>(c.coef);
  ResidFFParams prm{};
  for (int i = 0; i < 3; ++i) {
    prm.fields[i] = Ein[i];
    prm.fields[3 + i] = Hin[3 + i];
    prm.fields[6 + i] = Estar[i];
    prm.out[i] = R[i];
  }
  prm.coef[CF_A] = cf[0];
  prm.coef[CF_B] = cf[1];
  prm.coef[CF_C] = cf[2];
  for (int d = 0; d < 3; ++d)
    for (int o = 0; o < 4; ++o) prm.band[d][o] = bandff(c, d, o);
  int n = e_terms(half, prm.terms);
  for (int k = 0; k < 3; ++k) {
    Term t{};
    t.field = 6 + k;
    t.out = k;
    t.op[0] = t.op[1] = t.op[2] = OP_M;
    t.coef = CF_ONE;
    t.sign = -1.f;
    prm.terms[n++] = t;
    t.op[kStiffDir[half - 1][k]] = OP_S;
    t.coef = CF_C;
    prm.terms[n++] = t;
  }
  prm.nterms = n;
  prm.Nx = c.N[0];
  prm.Ny = c.N[1];
  prm.Nz = c.N[2];
  prm.pitch = c.pitch;
  prm.src_comp = (c.src_comp >= 0 && c.src_amp != 0.0) ? c.src_comp : -1;
  for (int d = 0; d < 3; ++d) {
    prm.src_i0[d] = c.src_i0[d];
    for (int q = 0; q <= kMaxP; ++q) prm.src_w[d][q] = c.src_w[d][q];
  }
  prm.src_amp = c.src_amp;
  prm.src_f0 = c.src_f0;
  prm.src_t0 = c.src_t0;
  prm.src_s = c.src_s;
  prm.tau = c.dt;
  prm.t_frac = half == 1 ? 0.25 : 0.75;
  prm.clock_t0 = c.d_clock_t0;
  prm.clock_step = c.d_clock_step;
  dim3 grid((c.N[0] + 31) / 32, (c.N[1] + 7) / 8, (c.N[2] + 7) / 8);
  prof_begin(c, "resid_Eff", (double)c.Nc * 4.0 * 15.0);  // reads 9 fields + a, b, c, writes 3
  resid_ff_kernel<P><<<grid, dim3(32, 8), resid_ff_smem<P>(), c.stream>>>(prm);
  prof_end(c);
  return cudaGetLastError();
}

// Right-hand side with the material inside the integrals (rhs_quad): zero the
// outputs, then one launch over tiles of 8^3 elements.  fields / terms as for
// rhs_kernel; the source (E half steps) with b of the element holding it.
template <typename T, int P>
cudaError_t launch_rhs_quad(Ctx& c, const T* const* fields, int nfields, T* const* out, const Term* terms,
                            int nterms, bool source, double t_frac) {
  QuadParams<T> prm{};
  for (int i = 0; i < nfields; ++i) prm.fields[i] = fields[i];
  for (int i = 0; i < 3; ++i) {
    prm.out[i] = out[i];
    cudaError_t e = cudaMemsetAsync(out[i], 0, c.Np * sizeof(T), c.stream);
    if (e != cudaSuccess) return e;
  }
  const T* tq = reinterpret_cast<const T*>(c.tabq);
  size_t off = 0;
  for (int d = 0; d < 3; ++d) {
    prm.loc[d] = tq + off;
    off += (size_t)c.n[d] * 4 * (P + 1) * (P + 1);
    prm.n[d] = c.n[d];
  }
  prm.eps = c.d_eps;
  prm.mu = c.d_mu;
  prm.sigma = c.d_sigma;
  prm.tau = c.dt;
  for (int k = 0; k < nterms; ++k) prm.terms[k] = terms[k];
  prm.nterms = nterms;
  prm.Nx = c.N[0];
  prm.Ny = c.N[1];
  prm.Nz = c.N[2];
  prm.pitch = c.pitch;
  prm.src_comp = (source && c.src_comp >= 0 && c.src_amp != 0.0) ? c.src_comp : -1;
  for (int d = 0; d < 3; ++d) {
    prm.src_e[d] = c.src_i0[d];
    for (int q = 0; q <= kMaxP; ++q) prm.src_w[d][q] = T(c.src_w[d][q]);
  }
  prm.src_amp = c.src_amp;
  prm.src_f0 = c.src_f0;
  prm.src_t0 = c.src_t0;
  prm.src_s = c.src_s;
  prm.t_frac = t_frac;
  prm.clock_t0 = c.d_clock_t0;
  prm.clock_step = c.d_clock_step;
  dim3 grid((c.n[0] + 7) / 8, (c.n[1] + 7) / 8, (c.n[2] + 7) / 8);
  if constexpr (sizeof(T) == 8 && P > 3) {  // the FP64 tiles of p >= 4 do not fit in shared memory
    return cudaErrorInvalidValue;          // (adi_create rejects that combination)
  } else {
    prof_begin(c, "rhs_quad", (double)c.Nc * sizeof(T) * (nfields + 3));
    rhs_quad_kernel<T, P><<<grid, 512, QuadTile<T, P>::bytes(nfields), c.stream>>>(prm, nfields);
    prof_end(c);
    return cudaGetLastError();
  }
}

// Right-hand side of an E half step (eqs. discrete1 / discrete3) into c.rhs.
template <typename T, int P>
cudaError_t e_rhs(Ctx& c, int half) {
  T** cur = reinterpret_cast<T**>(c.cur);
  T** hlf = reinterpret_cast<T**>(c.half);
  T** R = reinterpret_cast<T**>(c.rhs);
  T** cf = reinterpret_cast<T**>(c.coef);
  T* const* Ein = half == 1 ? cur : hlf;
  T* const* Hin = cur;  // H^n (half 1) or H^{n+1/2} (half 2), updated in place
  RhsParams<T> prm{};
  for (int i = 0; i < 3; ++i) {
    prm.fields[i] = Ein[i];
    prm.fields[3 + i] = Hin[3 + i];
    prm.out[i] = R[i];
  }
  prm.nfields = 6;
  prm.coef[CF_A] = cf[0];
  prm.coef[CF_B] = cf[1];
  prm.coef[CF_C] = cf[2];
  prm.coef[CF_D] = nullptr;
  for (int d = 0; d < 3; ++d) prm.ax[d] = axis_dev<T>(c, d);
  prm.nterms = e_terms(half, prm.terms);
  prm.Nx = c.N[0];
  prm.Ny = c.N[1];
  prm.Nz = c.N[2];
  prm.pitch = c.pitch;
  prm.src_comp = (c.src_comp >= 0 && c.src_amp != 0.0) ? c.src_comp : -1;
  for (int d = 0; d < 3; ++d) {
    prm.src_i0[d] = c.src_i0[d];
    for (int q = 0; q <= kMaxP; ++q) prm.src_w[d][q] = T(c.src_w[d][q]);
  }
  prm.src_amp = c.src_amp;
  prm.src_f0 = c.src_f0;
  prm.src_t0 = c.src_t0;
  prm.src_s = c.src_s;
  prm.tau = c.dt;
  prm.t_frac = half == 1 ? 0.25 : 0.75;
  prm.clock_t0 = c.d_clock_t0;
  prm.clock_step = c.d_clock_step;
  prm.advance_clock = 0;
  double bytes = (double)c.Nc * sizeof(T) * 12.0;
  const bool mixed = c.precision == ADI_PREC_MIXED;
  return c.rhs_quad ? launch_rhs_quad<T, P>(c, prm.fields, 6, R, prm.terms, prm.nterms, true, prm.t_frac)
                    : launch_rhs_e<T, P>(c, prm, half, bytes, mixed);
}

// E half step: the right-hand side, then the line solves (e_solve), then in
// mixed precision one refinement.
template <typename T, int P>
cudaError_t e_substep(Ctx& c, int half) {
  T** cur = reinterpret_cast<T**>(c.cur);
  T** hlf = reinterpret_cast<T**>(c.half);
  T** R = reinterpret_cast<T**>(c.rhs);
  T* const* Ein = half == 1 ? cur : hlf;
  T* const* Hin = cur;
  T* const* Eout = half == 1 ? hlf : cur;
  const bool mixed = c.precision == ADI_PREC_MIXED;
  cudaError_t e = e_rhs<T, P>(c, half);
  if (e != cudaSuccess) return e;
  e = e_solve<T, P>(c, half, R, Eout);
  if (e != cudaSuccess || !mixed || !c.mixed_refine) return e;
  if constexpr (sizeof(T) == 4) {
    // one refinement: R = RHS - T E* in FP64, T delta = R in place, E = E* + delta
    e = c.mixed_fp64_residual ? launch_resid<P>(c, half, Ein, Hin, Eout, R)
                              : launch_resid_ff<P>(c, half, Ein, Hin, Eout, R);
    if (e == cudaSuccess) e = e_solve<T, P>(c, half, R, R);
    if (e == cudaSuccess) {
      const long long rows = (long long)c.N[1] * c.N[2];
      prof_begin(c, "add_delta", (double)c.Nc * 4.0 * 9.0);
      add_delta_kernel<<<grid_for(rows * c.N[0], 256), 256, 0, c.stream>>>(Eout[0], Eout[1], Eout[2], R[0], R[1], R[2],
                                                                          c.N[0], c.pitch, rows);
      prof_end(c);
      e = cudaGetLastError();
    }
  }
  return e;
}

// H half step, general material: M H_new = M H_old - d C1 E_alpha + d C2 E_beta
// (eqs. discrete2 / discrete4), then three mass solves per component (H_i
// constrained in direction i).
template <typename T, int P>
cudaError_t h_substep_general(Ctx& c, int half) {
  T** cur = reinterpret_cast<T**>(c.cur);
  T** hlf = reinterpret_cast<T**>(c.half);
  T** R = reinterpret_cast<T**>(c.rhs);
  T** cf = reinterpret_cast<T**>(c.coef);
  RhsParams<T> prm{};
  // H lives in one buffer (cur) and is replaced by the new level:
  // alpha = E^n (half 1) or E^{n+1} (half 2) in cur, beta = E^{n+1/2} in half
  T* const* Hold = cur;
  T* const* Hout = cur;
  for (int i = 0; i < 3; ++i) {
    prm.fields[i] = Hold[3 + i];
    prm.fields[3 + i] = cur[i];
    prm.fields[6 + i] = hlf[i];
    prm.out[i] = R[i];
  }
  prm.nfields = 9;
  prm.coef[CF_D] = cf[3];
  for (int d = 0; d < 3; ++d) prm.ax[d] = axis_dev<T>(c, d);
  prm.nterms = h_terms(prm.terms);
  prm.Nx = c.N[0];
  prm.Ny = c.N[1];
  prm.Nz = c.N[2];
  prm.pitch = c.pitch;
  prm.src_comp = -1;
  prm.clock_t0 = c.d_clock_t0;
  prm.clock_step = c.d_clock_step;
  prm.advance_clock = half == 2 ? 1 : 0;
  double bytes = (double)c.Nc * sizeof(T) * 13.0;
  cudaError_t e;
  if (c.rhs_quad) {  // the clock advances in its own launch (the quad kernel does not touch it)
    e = launch_rhs_quad<T, P>(c, prm.fields, 9, R, prm.terms, prm.nterms, false, 0.0);
    if (e == cudaSuccess && half == 2) e = advance_clock(c);
  } else {
    e = launch_rhs<T, P>(c, prm, "rhs_H", bytes);
  }
  if (e != cudaSuccess) return e;
  static const char* mass_name[3] = {"line_x_mass", "line_y_mass", "line_z_mass"};
  for (int d = 0; d < 3; ++d) {
    LineJobs<T> js{};
    for (int i = 0; i < 3; ++i) js.job[i] = job_of<T>(R[i], d == 2 ? Hout[3 + i] : R[i], nullptr, 0.0, d == i);
    e = launch_line<T, P>(c, d, LM_MASS, js, 3, mass_name[d]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// H half step when mu is uniform (d constant): since the H system matrix is the
// 3D mass matrix, H_new = H_old + d M^-1 (-C1 E_alpha + C2 E_beta) exactly, and
// M^-1 (M (x) A (x) M) reduces to the 1D derivative D = M^-1 A along one axis
// (the other two factors cancel; the boundary constraints of E and H make the
// cancelled factors identical).  Componentwise:
//   H1 += d (-D_y E3_alpha + D_z E2_beta)
//   H2 += d (-D_z E1_alpha + D_x E3_beta)
//   H3 += d (-D_x E2_alpha + D_y E1_beta)
// done as three axis passes (z, x, y), two components each.  Every pass adds to
// an H component that another pass also adds to, so the passes run in order.
template <typename T, int P>
cudaError_t h_substep_uniform(Ctx& c, int half) {
  T** cur = reinterpret_cast<T**>(c.cur);
  T** hlf = reinterpret_cast<T**>(c.half);
  T* const* H = cur + 3;  // H is updated in place (H^n is dead once H^{n+1/2} exists)
  T* const* Ea = cur;     // alpha: E^n (half 1) or E^{n+1} (half 2)
  T* const* Eb = hlf;     // beta:  E^{n+1/2}
  const double d = c.d_uniform;
  // the staged y / z derivative kernel and the x kernel need no intermediate array
  LineJobs<T> js{};
  js.job[0] = job_of<T>(Eb[1], H[0], nullptr, d, 0);
  js.job[1] = job_of<T>(Ea[0], H[1], nullptr, -d, 0);
  cudaError_t e = launch_line<T, P>(c, 2, LM_DERIV, js, 2, "line_z_deriv");
  if (e != cudaSuccess) return e;
  js.job[0] = job_of<T>(Eb[2], H[1], nullptr, d, 0);
  js.job[1] = job_of<T>(Ea[1], H[2], nullptr, -d, 0);
  e = launch_line<T, P>(c, 0, LM_DERIV, js, 2, "line_x_deriv");
  if (e != cudaSuccess) return e;
  js.job[0] = job_of<T>(Ea[2], H[0], nullptr, -d, 0);
  js.job[1] = job_of<T>(Eb[0], H[2], nullptr, d, 0);
  e = launch_line<T, P>(c, 1, LM_DERIV, js, 2, "line_y_deriv");
  if (e != cudaSuccess) return e;
  if (half == 2) e = advance_clock(c);
  return e;
}

template <typename T, int P>
cudaError_t h_substep(Ctx& c, int half) {
  return c.mu_uniform ? h_substep_uniform<T, P>(c, half) : h_substep_general<T, P>(c, half);
}

// Inverse pivots of the row-scaled M + c S along each axis (Dirichlet-reduced,
// as every stiffness solve of the E half steps); they depend only on c, i.e.
// on the material and tau, so they are computed once by adi_factor.
template <typename T, int P>
cudaError_t pivots_tp(Ctx& c) {
  T** cf = reinterpret_cast<T**>(c.coef);
  static const char* name[3] = {"pivots_x", "pivots_y", "pivots_z"};
  for (int d = 0; d < 3; ++d) {
    if (!c.pivots[d]) {
      cudaError_t e = cudaMalloc(&c.pivots[d], c.Np * sizeof(T));
      if (e != cudaSuccess) return e;
    }
    LineJobs<T> js{};
    js.job[0] = job_of<T>(nullptr, reinterpret_cast<T*>(c.pivots[d]), cf[2], 0.0, 1);
    for (int m = 0; m < 2 * P; ++m) {  // the stiffness solves of every axis read the row factors
      if (!c.stiff_fac[d][m]) {
        cudaError_t e = cudaMalloc(&c.stiff_fac[d][m], c.Np * sizeof(T));
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c.stiff_fac[d][m], 0, c.Np * sizeof(T), c.stream);
        if (e != cudaSuccess) return e;
      }
      js.job[0].fac[m] = reinterpret_cast<T*>(c.stiff_fac[d][m]);
    }
    cudaError_t e = launch_line<T, P>(c, d, LM_PIVOT, js, 1, name[d]);
    if (e != cudaSuccess) return e;
  }
  return cudaStreamSynchronize(c.stream);
}

template <typename T, int P>
cudaError_t substep_tp(Ctx& c, int which) {
  switch (which) {
    case 0: return e_substep<T, P>(c, 1);
    case 1: return h_substep<T, P>(c, 1);
    case 2: return e_substep<T, P>(c, 2);
    case 3: return h_substep<T, P>(c, 2);
    default: {  // 4, 5: half step 1 or 2, E then H
      const int half = which - 3;
      cudaError_t e = e_substep<T, P>(c, half);
      return e == cudaSuccess ? h_substep<T, P>(c, half) : e;
    }
  }
}

template <typename T>
cudaError_t substep_t(Ctx& c, int which) {
  switch (c.p) {
    case 1: return substep_tp<T, 1>(c, which);
    case 2: return substep_tp<T, 2>(c, which);
    case 3: return substep_tp<T, 3>(c, which);
    default: return substep_tp<T, 4>(c, which);
  }
}

// Opt in to large dynamic shared memory once, outside any stream capture:
// the per-block opt-in limit minus the kernel's static shared memory.
template <typename K>
cudaError_t opt_in(K kern, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <typename T, int P>
cudaError_t prepare_tp(int optin) {
  cudaError_t e = opt_in(rhs_kernel<T, P, 32, 8, 8>, optin);
  if (e == cudaSuccess) e = opt_in(line_xws_kernel<T, P>, optin);
  if (e == cudaSuccess) e = opt_in(rhs_e_kernel<T, P, 1>, optin);
  if (e == cudaSuccess) e = opt_in(rhs_e_kernel<T, P, 2>, optin);
  if constexpr (sizeof(T) == 4) {
    if (e == cudaSuccess) e = opt_in(line_xw_kernel<P, LM_MASS>, optin);
    if (e == cudaSuccess) e = opt_in(line_xw_kernel<P, LM_DERIV>, optin);
    if (e == cudaSuccess) e = opt_in(rhs_e_mma_kernel<P>, optin);
    if (e == cudaSuccess) e = opt_in(resid_kernel<P>, optin);
    if (e == cudaSuccess) e = opt_in(resid_ff_kernel<P>, optin);
  }
  if constexpr (!(sizeof(T) == 8 && P > 3))
    if (e == cudaSuccess) e = opt_in(rhs_quad_kernel<T, P>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_MASS, true>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_STIFF, true>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_DERIV, true>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_PIVOT, true>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_PIVOT, false>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_MASS, false>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_STIFF, false>, optin);
  if (e == cudaSuccess) e = opt_in(line_kernel<T, P, LM_DERIV, false>, optin);
  return e;
}

template <typename T>
cudaError_t prepare_t(int p, int optin) {
  switch (p) {
    case 1: return prepare_tp<T, 1>(optin);
    case 2: return prepare_tp<T, 2>(optin);
    case 3: return prepare_tp<T, 3>(optin);
    default: return prepare_tp<T, 4>(optin);
  }
}

// ------------------------------------------------------------ diagnostics
// Norms of the state as functions on the unit cube (the paper's L2 and H1 norms
// of E and H over time in the head experiment, Figure head_norms, and the L2 /
// H(curl) norms of its manufactured-solution errors).  Each squared norm is a
// quadratic form of the Kronecker 1D matrices: for coefficients c of one
// component, int u^2 = c . (M(x)M(x)M) c and int |grad u|^2 =
// c . (S(x)M(x)M + M(x)S(x)M + M(x)M(x)S) c; int |curl u|^2 adds, for each curl
// component (d_a u_b - d_b u_a), the two squares and minus twice the cross
// term, e.g. int d2 u3 d3 u2 = u2 . (M(x)A(x)B) u3 (A: derivative on the trial,
// B on the test function).  The generic right-hand-side kernel applies the
// terms into the scratch arrays; dot3_kernel forms sum_i c_i . (K c)_i in FP64.
template <typename T>
__global__ void dot3_kernel(const T* __restrict__ a0, const T* __restrict__ a1, const T* __restrict__ a2,
                            const T* __restrict__ b0, const T* __restrict__ b1, const T* __restrict__ b2, int Nx,
                            int pitch, long long rows, double* out) {
  __shared__ double part[32];
  double s = 0.0;
  const long long n = rows * Nx;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    const long long o = (g / Nx) * pitch + (g % Nx);
    s += (double)a0[o] * (double)b0[o] + (double)a1[o] * (double)b1[o] + (double)a2[o] * (double)b2[o];
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

// Values of one coefficient array on a uniform grid of a plane: per output
// point the (p+1)^3 B-splines that are nonzero there, from host tables
// tab[axis][point] = (first index, p+1 values) of the three 1D point sets.
template <typename T>
__global__ void plane_kernel(const T* __restrict__ u, int Ny, int pitch, int p, int axis, int nu, int nv,
                             const double* __restrict__ tab, double* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nu * nv) return;
  const int j = idx % nu, k = idx / nu;
  const int rec = p + 2;
  const double* t0 = tab;                      // the plane's own coordinate (one point)
  const double* tu = tab + rec;                // nu points
  const double* tv = tab + rec * (1 + nu);     // nv points
  // per axis x, y, z: the record of this output point
  const double* r[3];
  const int o0 = axis == 0 ? 1 : 0;            // first of the two in-plane axes
  const int o1 = axis == 2 ? 1 : 2;
  r[axis] = t0;
  r[o0] = tu + (long long)j * rec;
  r[o1] = tv + (long long)k * rec;
  const int ix = (int)r[0][0], iy = (int)r[1][0], iz = (int)r[2][0];
  double v = 0.0;
  for (int cz = 0; cz <= p; ++cz)
    for (int cy = 0; cy <= p; ++cy) {
      const double wyz = r[2][1 + cz] * r[1][1 + cy];
      const T* row = u + ((long long)(iz + cz) * Ny + (iy + cy)) * pitch + ix;
      for (int cx = 0; cx <= p; ++cx) v += wyz * r[0][1 + cx] * (double)row[cx];
    }
  out[idx] = v;
}

template <typename T, int P>
cudaError_t norms_tp(Ctx& c, double* d_acc) {
  T** cur = reinterpret_cast<T**>(c.cur);
  T** R = reinterpret_cast<T**>(c.rhs);
  auto term = [](int field, int out, int ox, int oy, int oz, float sign) {
    Term t{};
    t.field = field;
    t.out = out;
    t.op[0] = ox;
    t.op[1] = oy;
    t.op[2] = oz;
    t.coef = CF_ONE;
    t.sign = sign;
    return t;
  };
  const long long rows = (long long)c.N[1] * c.N[2];
  for (int g = 0; g < 2; ++g) {  // E, then H
    RhsParams<T> prm{};
    for (int i = 0; i < 3; ++i) {
      prm.fields[i] = cur[3 * g + i];
      prm.out[i] = R[i];
    }
    prm.nfields = 3;
    for (int k = 0; k < 5; ++k) prm.coef[k] = nullptr;
    for (int d = 0; d < 3; ++d) prm.ax[d] = axis_dev<T>(c, d);
    prm.Nx = c.N[0];
    prm.Ny = c.N[1];
    prm.Nz = c.N[2];
    prm.pitch = c.pitch;
    prm.src_comp = -1;
    prm.clock_t0 = c.d_clock_t0;
    prm.clock_step = c.d_clock_step;
    prm.advance_clock = 0;
    for (int form = 0; form < 3; ++form) {
      int n = 0;
      if (form == 0) {          // int u_i^2
        for (int i = 0; i < 3; ++i) prm.terms[n++] = term(i, i, OP_M, OP_M, OP_M, 1.f);
      } else if (form == 1) {   // int |grad u_i|^2
        for (int i = 0; i < 3; ++i) {
          prm.terms[n++] = term(i, i, OP_S, OP_M, OP_M, 1.f);
          prm.terms[n++] = term(i, i, OP_M, OP_S, OP_M, 1.f);
          prm.terms[n++] = term(i, i, OP_M, OP_M, OP_S, 1.f);
        }
      } else {                  // int |curl u|^2, terms grouped by the field they read
        prm.terms[n++] = term(0, 0, OP_M, OP_M, OP_S, 1.f);   // (d3 u1)^2
        prm.terms[n++] = term(0, 0, OP_M, OP_S, OP_M, 1.f);   // (d2 u1)^2
        prm.terms[n++] = term(0, 2, OP_B, OP_M, OP_A, -2.f);  // -2 d3 u1 d1 u3
        prm.terms[n++] = term(1, 1, OP_M, OP_M, OP_S, 1.f);   // (d3 u2)^2
        prm.terms[n++] = term(1, 1, OP_S, OP_M, OP_M, 1.f);   // (d1 u2)^2
        prm.terms[n++] = term(1, 0, OP_A, OP_B, OP_M, -2.f);  // -2 d1 u2 d2 u1
        prm.terms[n++] = term(2, 2, OP_M, OP_S, OP_M, 1.f);   // (d2 u3)^2
        prm.terms[n++] = term(2, 2, OP_S, OP_M, OP_M, 1.f);   // (d1 u3)^2
        prm.terms[n++] = term(2, 1, OP_M, OP_A, OP_B, -2.f);  // -2 d2 u3 d3 u2
      }
      prm.nterms = n;
      cudaError_t e = launch_rhs<T, P>(c, prm, "norm_form", (double)c.Nc * sizeof(T) * 6.0);
      if (e != cudaSuccess) return e;
      dot3_kernel<T><<<grid_for(rows * c.N[0], 256), 256, 0, c.stream>>>(
          prm.fields[0], prm.fields[1], prm.fields[2], R[0], R[1], R[2], c.N[0], c.pitch, rows, d_acc + 2 * form + g);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t norms_t(Ctx& c, double* d_acc) {
  switch (c.p) {
    case 1: return norms_tp<T, 1>(c, d_acc);
    case 2: return norms_tp<T, 2>(c, d_acc);
    case 3: return norms_tp<T, 3>(c, d_acc);
    default: return norms_tp<T, 4>(c, d_acc);
  }
}

template <typename T>
cudaError_t plane_t(Ctx& c, int comp, int axis, int nu, int nv, const double* d_tab, double* d_out) {
  const int n = nu * nv;
  plane_kernel<T><<<(n + 255) / 256, 256, 0, c.stream>>>(reinterpret_cast<const T*>(c.cur[comp]), c.N[1], c.pitch,
                                                          c.p, axis, nu, nv, d_tab, d_out);
  return cudaGetLastError();
}

unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 64) b = 152LL * 64;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

template <typename T>
cudaError_t pivots_t(Ctx& c) {
  switch (c.p) {
    case 1: return pivots_tp<T, 1>(c);
    case 2: return pivots_tp<T, 2>(c);
    case 3: return pivots_tp<T, 3>(c);
    default: return pivots_tp<T, 4>(c);
  }
}

// This file is compiled twice: with ADI_KERNELS_F64 it holds the FP64 step, else
// the FP32 / mixed step and everything shared; the two halves build in parallel.
// The element-type-specific entry points are named *_f32 / *_f64; the
// dispatchers below pick one by c.precision.
#ifdef ADI_KERNELS_F64
cudaError_t upload_tables_f64(Ctx& c, int optin) {
  cudaError_t e = prepare_t<double>(c.p, optin);
  if (e == cudaSuccess) e = upload_tables_t<double>(c);
  if (e == cudaSuccess && c.rhs_quad) e = upload_quad_tables<double>(c);
  if (e == cudaSuccess) e = pivots_t<double>(c);
  return e;
}
cudaError_t run_substep_f64(Ctx& c, int which) { return substep_t<double>(c, which); }
cudaError_t norms_f64(Ctx& c, double* d_acc) { return norms_t<double>(c, d_acc); }
cudaError_t plane_f64(Ctx& c, int comp, int axis, int nu, int nv, const double* d_tab, double* d_out) {
  return plane_t<double>(c, comp, axis, nu, nv, d_tab, d_out);
}
#else
cudaError_t upload_tables_f64(Ctx& c, int optin);
cudaError_t run_substep_f64(Ctx& c, int which);
cudaError_t norms_f64(Ctx& c, double* d_acc);
cudaError_t plane_f64(Ctx& c, int comp, int axis, int nu, int nv, const double* d_tab, double* d_out);

cudaError_t field_norms_dev(Ctx& c, double* d_acc) {
  cudaError_t e = cudaMemsetAsync(d_acc, 0, 6 * sizeof(double), c.stream);
  if (e != cudaSuccess) return e;
  return c.precision == ADI_PREC_FP64 ? norms_f64(c, d_acc) : norms_t<float>(c, d_acc);
}

cudaError_t plane_dev(Ctx& c, int comp, int axis, int nu, int nv, const double* d_tab, double* d_out) {
  return c.precision == ADI_PREC_FP64 ? plane_f64(c, comp, axis, nu, nv, d_tab, d_out)
                                      : plane_t<float>(c, comp, axis, nu, nv, d_tab, d_out);
}

cudaError_t upload_tables(Ctx& c) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device);
  if (e != cudaSuccess) return e;
  c.smem_optin = optin;
  if (c.precision == ADI_PREC_FP64) return upload_tables_f64(c, optin);
  e = prepare_t<float>(c.p, optin);
  if (e != cudaSuccess) return e;
  e = upload_tables_t<float>(c);
  if (e == cudaSuccess && c.rhs_quad) e = upload_quad_tables<float>(c);
  if (e != cudaSuccess) return e;
  if (c.precision == ADI_PREC_MIXED) {  // FP64 bands for the residual: per axis M, S, A, B
    std::vector<double> h;
    for (int d = 0; d < 3; ++d) {
      const Axis1D& ax = c.axes[d];
      for (const std::vector<double>* v : {&ax.M, &ax.S, &ax.A, &ax.B}) h.insert(h.end(), v->begin(), v->end());
    }
    if (!c.tab64) {
      e = cudaMalloc((void**)&c.tab64, h.size() * sizeof(double));
      if (e != cudaSuccess) return e;
      c.tab64_bytes = h.size() * sizeof(double);
    }
    e = cudaMemcpyAsync(c.tab64, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream);
    // the same tables as float pairs hi + lo (hi = the nearest float, lo = the nearest float of the rest)
    std::vector<float2> hf(h.size());
    for (size_t i = 0; i < h.size(); ++i) {
      const float hi = (float)h[i];
      hf[i] = make_float2(hi, (float)(h[i] - (double)hi));
    }
    if (e == cudaSuccess && !c.tabff) e = cudaMalloc((void**)&c.tabff, hf.size() * sizeof(float2));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c.tabff, hf.data(), hf.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return e;
  }
  return pivots_t<float>(c);
}

cudaError_t run_substep(Ctx& c, int which) {
  return c.precision == ADI_PREC_FP64 ? run_substep_f64(c, which) : substep_t<float>(c, which);
}

cudaError_t run_step(Ctx& c) {
  cudaError_t e = run_substep(c, 4);
  return e == cudaSuccess ? run_substep(c, 5) : e;
}

// 16-byte accesses when the dense array starts on a 16-byte boundary
template <typename S, typename T>
void launch_set(Ctx& c, const S* d_src, void* const* dst, int* d_bad) {
  constexpr int V = 16 / sizeof(S);
  T* const* d = reinterpret_cast<T* const*>(dst);
  const long long n = 6LL * (long long)c.Nc;
  if ((reinterpret_cast<uintptr_t>(d_src) & 15) == 0) {
    set_fields_kernel<S, T, V><<<grid_for(n / V + V, 256), 256, 0, c.stream>>>(
        d_src, d[0], d[1], d[2], d[3], d[4], d[5], c.N[0], c.N[1], c.N[2], c.pitch, d_bad);
  } else {
    set_fields_kernel<S, T, 1><<<grid_for(n, 256), 256, 0, c.stream>>>(d_src, d[0], d[1], d[2], d[3], d[4], d[5], c.N[0],
                                                                       c.N[1], c.N[2], c.pitch, d_bad);
  }
}
template <typename S, typename T>
void launch_get(Ctx& c, S* d_dst, int* d_bad) {
  constexpr int V = 16 / sizeof(S);
  T** s = reinterpret_cast<T**>(c.cur);
  const long long n = 6LL * (long long)c.Nc;
  if ((reinterpret_cast<uintptr_t>(d_dst) & 15) == 0) {
    get_fields_kernel<S, T, V><<<grid_for(n / V + V, 256), 256, 0, c.stream>>>(
        d_dst, s[0], s[1], s[2], s[3], s[4], s[5], c.N[0], c.N[1], c.N[2], c.pitch, d_bad);
  } else {
    get_fields_kernel<S, T, 1><<<grid_for(n, 256), 256, 0, c.stream>>>(d_dst, s[0], s[1], s[2], s[3], s[4], s[5], c.N[0],
                                                                       c.N[1], c.N[2], c.pitch, d_bad);
  }
}

template <typename S>
cudaError_t set_fields_into(Ctx& c, const S* d_src, void* const* dst, int* d_bad) {
  if (c.precision == ADI_PREC_FP64) launch_set<S, double>(c, d_src, dst, d_bad);
  else launch_set<S, float>(c, d_src, dst, d_bad);
  return cudaGetLastError();
}
template cudaError_t set_fields_into<double>(Ctx&, const double*, void* const*, int*);
template cudaError_t set_fields_into<float>(Ctx&, const float*, void* const*, int*);

template <typename S>
cudaError_t set_fields_dev(Ctx& c, const S* d_src) {
  return set_fields_into<S>(c, d_src, c.cur, nullptr);
}
template cudaError_t set_fields_dev<double>(Ctx&, const double*);
template cudaError_t set_fields_dev<float>(Ctx&, const float*);

template <typename S>
cudaError_t check_finite_dev(Ctx& c, const S* d_src, long long n, int* d_bad) {
  finite_kernel<S><<<grid_for(n, 256), 256, 0, c.stream>>>(d_src, n, d_bad);
  return cudaGetLastError();
}
template cudaError_t check_finite_dev<double>(Ctx&, const double*, long long, int*);
template cudaError_t check_finite_dev<float>(Ctx&, const float*, long long, int*);

template <typename S>
cudaError_t get_fields_dev(Ctx& c, S* d_dst, int* d_bad) {
  if (c.precision == ADI_PREC_FP64) launch_get<S, double>(c, d_dst, d_bad);
  else launch_get<S, float>(c, d_dst, d_bad);
  return cudaGetLastError();
}
template cudaError_t get_fields_dev<double>(Ctx&, double*, int*);
template cudaError_t get_fields_dev<float>(Ctx&, float*, int*);

cudaError_t make_tensor_maps(Ctx& c) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  EncodeTiledFn enc = reinterpret_cast<EncodeTiledFn>(fn);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = encode_map(c, enc, c.cur[i], &c.tmap_cur[i]);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = encode_map(c, enc, c.half[i], &c.tmap_half[i]);
  c.tmaps_ok = e == cudaSuccess;
  return e;
}

cudaError_t wait_selftest(Ctx& c, int which, int budget) {
  wait_selftest_kernel<<<1, 32, 0, c.stream>>>(which, budget, c.d_err);
  return cudaGetLastError();
}

cudaError_t set_clock(Ctx& c, double t0) {
  clock_kernel<<<1, 1, 0, c.stream>>>(c.d_clock_t0, c.d_clock_step, t0);
  return cudaGetLastError();
}

cudaError_t commit_fields(Ctx& c, const int* bad, int* refused, double t) {
  CommitArgs a;
  void* scratch[6] = {c.rhs[0], c.rhs[1], c.rhs[2], c.half[0], c.half[1], c.half[2]};
  for (int i = 0; i < 6; ++i) {
    a.src[i] = reinterpret_cast<const uint4*>(scratch[i]);
    a.dst[i] = reinterpret_cast<uint4*>(c.cur[i]);
  }
  const long long n = (long long)(c.Np * c.esize / 16);  // pitch is a multiple of 4 elements
  commit_kernel<<<grid_for(6 * n, 256), 256, 0, c.stream>>>(a, n, bad, refused, c.d_clock_t0, c.d_clock_step, t);
  return cudaGetLastError();
}

cudaError_t compute_coefficients(Ctx& c) {
  const int p = c.p;
  std::vector<double> G;
  size_t offs[4] = {0, 0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    offs[d] = G.size();
    G.insert(G.end(), c.axes[d].G.begin(), c.axes[d].G.end());
  }
  double* dG = nullptr;
  unsigned long long* dmin = nullptr;
  cudaError_t e = cudaMalloc(&dG, G.size() * sizeof(double));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&dmin, sizeof(unsigned long long));
  if (e != cudaSuccess) { cudaFree(dG); return e; }
  unsigned long long init = 0x7FEFFFFFFFFFFFFFULL;  // largest finite double
  cudaMemcpyAsync(dG, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream);
  cudaMemcpyAsync(dmin, &init, sizeof(init), cudaMemcpyHostToDevice, c.stream);
  unsigned g = grid_for((long long)c.Nc, 256);
  if (c.precision == ADI_PREC_FP64) {
    double** cf = reinterpret_cast<double**>(c.coef);
    coef_kernel<double><<<g, 256, 0, c.stream>>>(c.d_eps, c.d_mu, c.d_sigma, dG + offs[0], dG + offs[1], dG + offs[2],
                                                c.n[0], c.n[1], c.n[2], p, c.pitch, c.dt, cf[0], cf[1], cf[2], cf[3], dmin);
  } else {
    float** cf = reinterpret_cast<float**>(c.coef);
    coef_kernel<float><<<g, 256, 0, c.stream>>>(c.d_eps, c.d_mu, c.d_sigma, dG + offs[0], dG + offs[1], dG + offs[2],
                                               c.n[0], c.n[1], c.n[2], p, c.pitch, c.dt, cf[0], cf[1], cf[2], cf[3], dmin);
  }
  e = cudaGetLastError();
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, dmin, sizeof(bits), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cudaFree(dG);
  cudaFree(dmin);
  if (e == cudaSuccess) {
    double m;
    memcpy(&m, &bits, sizeof(m));
    c.min_eps_mu = m;
  }
  return e;
}

#endif  // ADI_KERNELS_F64

}  // namespace adi
