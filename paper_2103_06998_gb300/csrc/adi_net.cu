// Learned coarse-step corrector (include/adi_corrector.h): a 4-layer 3x3x3
// convolution net on the coefficient grid, its training (gradients + Adam) and
// the guarded time loop.  The paper has no learned component; this follows the
// definitions in the header.
//
// Convolutions (forward and input gradient) are implicit GEMMs on the 5th
// generation tensor cores.  A CTA owns a work unit (x segment, 2 y lines, a chunk
// of z planes) and marches along z: each haloed z plane is one slot of a 4-slot
// ring in shared memory, loaded by 5D TMA boxes straight into the no-swizzle
// K-major core-matrix layout ([8-channel chunk][voxel row], 16-byte rows); for
// each of the 27 taps the A operand of tcgen05.mma is the slot of plane z+dz-1
// with its rows shifted by the tap's in-plane offset (M = 128 voxels, N = output
// channels, K = 16 channels per instruction).  Warp 0 issues loads and MMAs
// into two tensor-memory accumulator buffers; warps 4..7 read them back with
// tcgen05.ld for the fused epilogue (bias + ReLU, ReLU mask, or FP32 output).
// Weight gradients are reductions over all voxels on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/adi_corrector.h"
#include "adi_internal.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kCI[4] = {16, 32, 32, 32};  // padded input channels per layer
constexpr int kCO[4] = {32, 32, 32, 16};  // padded output channels per layer
constexpr int kTY = 4;                    // x-lines (y rows) per convolution block
constexpr int kXBMax = 130;               // widest x segment of a block
constexpr int kConvThreads = 256;
constexpr int kWgThreads = 288;
constexpr int kTmemCols = 512;  // two accumulator buffers of 256 columns

constexpr long long w_off(int l) {
  return l == 0 ? 0 : w_off(l - 1) + 27LL * kCI[l - 1] * kCO[l - 1] + kCO[l - 1];
}
constexpr long long b_off(int l) { return w_off(l) + 27LL * kCI[l] * kCO[l]; }
static_assert(w_off(4) == ADI_NET_PARAMS, "parameter layout");

enum Epi : int { EPI_RELU = 0, EPI_LINEAR = 1, EPI_MASK = 2 };

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit_wait() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start address,
// leading byte offset (between core matrices adjacent along K), stride byte
// offset (between 8-row groups), version 1 in bits 46-47.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int N>
__host__ __device__ constexpr uint32_t idesc_bf16_m128() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// bounded wait for phase `parity`; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = su32(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(slot)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(kTmemCols) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
               : "memory");
}

// 32 lanes x 16 / 32 consecutive 32-bit columns; warp-collective
__device__ __forceinline__ void tmem_ld16(uint32_t t, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(t));
}
__device__ __forceinline__ void tmem_ld32(uint32_t t, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(t));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// ------------------------------------------------------------ block geometry
// A block is (x segment, TY consecutive y, one z).  Haloed voxels are numbered
// row = xh + Xh (yh + Yh zh), xh in [0, XB+2), yh in [0, TY+2), zh in [0, 3);
// a tap (dz, dy, dx) shifts rows by (dx-1) + Xh ((dy-1) + Yh (dz-1)).
struct Geom {
  int X, Y, Z;
  int XB, nseg, nyb, nblocks;
  int Xh, Yh;
  int rs;      // first output row
  int ntiles;  // 128-row MMA tiles per block
  int rows;    // rows of one chunk plane in shared memory
};

inline Geom make_geom(int X, int Y, int Z) {
  Geom g{};
  g.X = X;
  g.Y = Y;
  g.Z = Z;
  g.nseg = (X + kXBMax - 1) / kXBMax;
  g.XB = (X + g.nseg - 1) / g.nseg;
  g.nyb = (Y + kTY - 1) / kTY;
  g.nblocks = g.nseg * g.nyb * Z;
  g.Xh = g.XB + 2;
  g.Yh = kTY + 2;
  g.rs = 1 + g.Xh * (1 + g.Yh);
  const int count = g.XB + g.Xh * (kTY - 1);
  g.ntiles = (count + 127) / 128;
  const int maxoff = 1 + g.Xh + g.Xh * g.Yh;
  g.rows = g.rs + 128 * g.ntiles + maxoff;
  return g;
}

template <int CIN, int COUT>
__host__ __device__ constexpr size_t conv_wbytes() {
  return 27ull * CIN * COUT * 2;
}

// Plane-ring geometry of the convolutions.  A work unit is (x segment, 2
// consecutive y, a chunk of z); the CTA marches along z.  Each z plane of the
// unit's haloed (X_b+2) x 4 voxel window is one ring slot in shared memory:
// CIN/8 chunk planes of RS rows of 16 bytes (8 channels), row = xh + Xh yh,
// exactly the box a 5D TMA load writes.  Output rows are rs .. rs+128 nt-1 of
// a slot; tap (dz, dy, dx) reads plane z+dz-1 at row offset (dx-1) + Xh (dy-1).
constexpr int kRTY = 2;     // y lines per unit
constexpr int kSlots = 4;   // planes z-1, z, z+1 in use, z+2 loading
struct Ring {
  int X, Y, Z;
  int XB, nseg, nyb, nzc, zc, units;
  int Xh, Yh, rs, ntiles, RS;
};

inline Ring make_ring(int X, int Y, int Z, int sms) {
  Ring r{};
  r.X = X;
  r.Y = Y;
  r.Z = Z;
  r.nseg = (X + kXBMax - 1) / kXBMax;
  r.XB = (X + r.nseg - 1) / r.nseg;
  r.nyb = (Y + kRTY - 1) / kRTY;
  r.Xh = r.XB + 2;
  r.Yh = kRTY + 2;
  r.rs = 1 + r.Xh;
  const int count = r.XB + r.Xh * (kRTY - 1);
  r.ntiles = (count + 127) / 128;
  r.RS = ((r.rs + 128 * r.ntiles + r.Xh + 1) + 7) / 8 * 8;  // 128-byte aligned chunk planes
  const int cols = r.nseg * r.nyb;
  int nzc = (8 * sms + cols - 1) / cols;  // about eight units per SM: a short last wave
  if (nzc < 1) nzc = 1;
  if (nzc > Z) nzc = Z;
  r.zc = (Z + nzc - 1) / nzc;
  r.nzc = (Z + r.zc - 1) / r.zc;
  r.units = cols * r.nzc;
  return r;
}
template <int CIN, int COUT>
inline size_t ring_smem(const Ring& r) {  // worst-case alignment of the base and of the slots included
  return 3072 + conv_wbytes<CIN, COUT>() + (size_t)kSlots * (CIN / 8) * r.RS * 16;
}

struct ConvArgs {
  const bf16* w;      // packed [27][CIN/8][COUT][8]
  const float* bias;  // [COUT] (RELU, LINEAR)
  const bf16* mask;   // [V][COUT] (MASK): output kept where mask > 0
  void* out;          // bf16 [V][COUT] (RELU, MASK) or float [V][8] (LINEAR)
  Ring r;
  int* err;
};

// 5D TMA load of one chunk plane: box (8 channels, 1 chunk, Xh, Yh, 1 plane)
__device__ __forceinline__ void tma_plane(const CUtensorMap* map, uint32_t dst, uint64_t* bar, int c, int x, int y,
                                          int z) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];\n" ::"r"(dst),
      "l"(map), "r"(0), "r"(c), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// Warp-specialised: warp 0 is the producer (lane 0 issues the TMA plane loads
// and the MMAs of each output plane into one of two tensor-memory accumulator
// buffers), warps 4..7 are the consumers (epilogue, one tensor-memory lane
// quarter each).  Hand-offs use mbarriers only: plane loaded (per slot), MMAs of
// a buffer done (tcgen05.commit), buffer read out (4 consumer arrivals).
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kConvThreads, 1) conv_kernel(const ConvArgs a, const __grid_constant__ CUtensorMap map) {
  constexpr int CH = CIN / 8;
  constexpr uint32_t IDESC = idesc_bf16_m128<COUT>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* lbar = reinterpret_cast<uint64_t*>(base);        // [kSlots] plane loaded
  uint64_t* done = reinterpret_cast<uint64_t*>(base + 64);   // [2] MMAs of a buffer complete
  uint64_t* freed = reinterpret_cast<uint64_t*>(base + 96);  // [2] buffer read out by the consumers
  uint32_t* tslot = reinterpret_cast<uint32_t*>(base + 128);
  uint8_t* sW = base + 1024;
  uint8_t* sA = base + ((1024 + conv_wbytes<CIN, COUT>() + 1023) & ~(size_t)1023);
  const uint32_t sW32 = su32(sW), sA32 = su32(sA);
  const Ring& g = a.r;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t slot_bytes = (uint32_t)(CH * g.RS * 16);
  const uint32_t plane_tx = (uint32_t)(CH * g.Xh * g.Yh * 16);

  if (warp == 0) tmem_alloc(tslot);
  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) mbar_init(&lbar[s]);
    mbar_init(&done[0]);
    mbar_init(&done[1]);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(su32(&freed[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(su32(&freed[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int i = tid; i < (int)(conv_wbytes<CIN, COUT>() / 16); i += kConvThreads)
    cp16(sW32 + 16 * i, reinterpret_cast<const uint8_t*>(a.w) + 16 * (size_t)i, 16);
  cp_commit_wait();
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // weights: generic writes, tensor-core reads
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int cols = g.nseg * g.nyb;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t lph[kSlots] = {0u, 0u, 0u, 0u};
      bool lpend[kSlots] = {false, false, false, false};
      uint32_t dph[2] = {0u, 0u}, fph[2] = {0u, 0u};
      bool used[2] = {false, false};
      bool ok = true;
      // A descriptor offsets (16-byte units) of the nine (dy, dx) taps and of tile j / step ks
      int off9[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) off9[t] = g.rs + (t % 3 - 1) + g.Xh * (t / 3 - 1);
      const uint64_t a0 = sdesc(sA32, (uint32_t)g.RS * 16u, 128u);
      const uint64_t b0 = sdesc(sW32, COUT * 16u, 128u);
      for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
        const int col = u % cols, zi = u / cols;
        const int x0 = (col % g.nseg) * g.XB, y0 = (col / g.nseg) * kRTY;
        const int za = zi * g.zc, zb = min(g.Z, za + g.zc);
        auto load = [&](int p) {
          const int s = (p - za + 1) & 3;
          lpend[s] = true;
          mbar_expect(&lbar[s], plane_tx);
          for (int c = 0; c < CH; ++c)
            tma_plane(&map, sA32 + (uint32_t)s * slot_bytes + (uint32_t)(c * g.RS * 16), &lbar[s], c, x0 - 1, y0 - 1, p);
        };
        for (int p = za - 1; p <= min(za + 2, zb); ++p) load(p);
        for (int z = za; z < zb && ok; ++z) {
          const int i = z - za;
          const int buf = z & 1;
          for (int d = i == 0 ? 0 : 2; d < 3 && ok; ++d) {  // new planes of this output plane
            const int s = (i + d) & 3;
            ok = mbar_wait(&lbar[s], lph[s]);
            if (ok) {
              lph[s] ^= 1u;
              lpend[s] = false;
            }
          }
          if (ok && used[buf]) {  // the consumers have read this buffer's previous plane
            ok = mbar_wait(&freed[buf], fph[buf]);
            fph[buf] ^= 1u;
          }
          if (!ok) break;
          used[buf] = true;
          tc_fence_after();
          uint64_t sd[3];
#pragma unroll
          for (int dz = 0; dz < 3; ++dz) sd[dz] = a0 + (uint64_t)(((i + dz) & 3) * (int)(slot_bytes >> 4));
          const uint32_t d0 = tmem + (uint32_t)buf * 256u;
          for (int j = 0; j < g.ntiles; ++j) {
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
              const uint64_t ad = sd[tap / 9] + (uint64_t)(off9[tap % 9] + 128 * j);
#pragma unroll
              for (int ks = 0; ks < CIN / 16; ++ks)
                mma_bf16(d0 + (uint32_t)(j * COUT), ad + (uint64_t)(2 * ks * g.RS),
                         b0 + (uint64_t)((tap * CH + 2 * ks) * COUT), IDESC, (tap | ks) != 0 ? 1u : 0u);
            }
          }
          mma_commit(&done[buf]);
          if (i > 0) {  // MMAs of plane z-1 done: the slot of plane z-2 takes plane z+2
            const int pb = buf ^ 1;
            ok = mbar_wait(&done[pb], dph[pb]);
            dph[pb] ^= 1u;
            if (ok && z + 2 <= zb) load(z + 2);
          }
        }
        if (ok) {  // the unit's last plane: its MMAs done before the slots are reused
          const int lb = (zb - 1) & 1;
          ok = mbar_wait(&done[lb], dph[lb]);
          dph[lb] ^= 1u;
        }
      }
      if (!ok) {
        atomicOr(a.err, 2);
        for (int s = 0; s < kSlots; ++s)  // copies still in flight land before the CTA leaves
          if (lpend[s]) mbar_wait(&lbar[s], lph[s]);
        mbar_wait(&done[0], dph[0]);
        mbar_wait(&done[1], dph[1]);
      }
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ------------------------------------------------------------ consumers
    const int q = warp & 3;
    float bias[COUT];  // in registers for the whole kernel
#pragma unroll
    for (int c = 0; c < COUT; ++c) bias[c] = EPI == EPI_MASK ? 0.0f : a.bias[c];
    uint32_t dph[2] = {0u, 0u};
    bool ok = true;
    for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
      const int col = u % cols, zi = u / cols;
      const int x0 = (col % g.nseg) * g.XB, y0 = (col / g.nseg) * kRTY;
      const int za = zi * g.zc, zb = min(g.Z, za + g.zc);
      for (int z = za; z < zb; ++z) {
        const int buf = z & 1;
        ok = mbar_wait(&done[buf], dph[buf]);
        dph[buf] ^= 1u;
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int j = 0; j < g.ntiles; ++j) {
          uint32_t r[32];
          const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * 256u + (uint32_t)(j * COUT);
          if (COUT == 32) tmem_ld32(taddr, r);
          else tmem_ld16(taddr, r);
          tmem_wait_ld();
          const int row = g.rs + 128 * j + 32 * q + lane;
          const int yh = row / g.Xh, xh = row - yh * g.Xh;
          const int x = x0 + xh - 1, y = y0 + yh - 1;
          if (!(yh >= 1 && yh <= kRTY && xh >= 1 && xh <= g.XB && x < g.X && y < g.Y)) continue;
          const size_t v = ((size_t)z * g.Y + y) * g.X + x;
          if (EPI == EPI_LINEAR) {
            float o[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) o[c] = c < 6 ? __uint_as_float(r[c]) + bias[c] : 0.0f;
            float4* dst = reinterpret_cast<float4*>(static_cast<float*>(a.out) + v * 8);
            dst[0] = make_float4(o[0], o[1], o[2], o[3]);
            dst[1] = make_float4(o[4], o[5], o[6], o[7]);
          } else {
            uint32_t pk[COUT / 2];
            if (EPI == EPI_RELU) {
#pragma unroll
              for (int c = 0; c < COUT / 2; ++c)
                pk[c] = pack_bf16(fmaxf(__uint_as_float(r[2 * c]) + bias[2 * c], 0.0f),
                                  fmaxf(__uint_as_float(r[2 * c + 1]) + bias[2 * c + 1], 0.0f));
            } else {
              const uint4* mk = reinterpret_cast<const uint4*>(a.mask + v * COUT);
#pragma unroll
              for (int c8 = 0; c8 < COUT / 8; ++c8) {
                const uint4 m = mk[c8];
                const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  const int c = 8 * c8 + 2 * k;
                  pk[c / 2] = pack_bf16(bf_lo(mw[k]) > 0.0f ? __uint_as_float(r[c]) : 0.0f,
                                        bf_hi(mw[k]) > 0.0f ? __uint_as_float(r[c + 1]) : 0.0f);
                }
              }
            }
            uint4* dst = reinterpret_cast<uint4*>(static_cast<bf16*>(a.out) + v * COUT);
#pragma unroll
            for (int c8 = 0; c8 < COUT / 8; ++c8)
              dst[c8] = make_uint4(pk[4 * c8], pk[4 * c8 + 1], pk[4 * c8 + 2], pk[4 * c8 + 3]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(&freed[buf])) : "memory");
      }
    }
    if (!ok && lane == 0) atomicOr(a.err, 2);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem);
  }
}

// ------------------------------------------------------------ weight gradients
// dw[tap][ci][co] = sum_v in[v + tap - 1][ci] g[v][co],  db[co] = sum_v g[v][co]
// Blocks are (x segment, one y, one z); each CTA accumulates its blocks in
// registers and writes one partial sum (reduced by wg_reduce_kernel).
struct WgArgs {
  const bf16* in;  // [V][CIN]
  const bf16* gr;  // [V][COUT]
  float* partial;  // [gridDim.x][27 CIN COUT + COUT]
  Geom g;          // XB, nseg of the convolution geometry
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgThreads, 1) wgrad_kernel(const WgArgs a) {
  constexpr int NP = 27 * CIN;
  constexpr int PPT = (NP + kWgThreads - 1) / kWgThreads;
  extern __shared__ uint8_t smem_raw[];
  const Geom& g = a.g;
  const int Xh = g.XB + 2;
  bf16* sIn = reinterpret_cast<bf16*>(smem_raw);            // [9 Xh][CIN]
  bf16* sG = sIn + 9 * Xh * CIN;                             // [XB][COUT]
  const int tid = threadIdx.x;
  float acc[PPT][COUT];
  int offs[PPT];
#pragma unroll
  for (int pp = 0; pp < PPT; ++pp) {
    const int p = tid + pp * kWgThreads;
    const int tap = p / CIN, ci = p - tap * CIN;
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    offs[pp] = p < NP ? (dx + Xh * (dy + 3 * dz)) * CIN + ci : 0;
#pragma unroll
    for (int c = 0; c < COUT; ++c) acc[pp][c] = 0.0f;
  }
  float bacc = 0.0f;
  const int nblk = g.nseg * g.Y * g.Z;
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int seg = b % g.nseg;
    const int t = b / g.nseg;
    const int y0 = t % g.Y, z0 = t / g.Y;
    const int x0 = seg * g.XB;
    __syncthreads();
    for (int line = 0; line < 9; ++line) {
      const int zh = line / 3, yh = line % 3;
      const int z = z0 - 1 + zh, y = y0 - 1 + yh;
      const bool lin = z >= 0 && z < g.Z && y >= 0 && y < g.Y;
      const bf16* src_line = a.in + ((size_t)z * g.Y + y) * (size_t)g.X * CIN;
      for (int i = tid; i < Xh * (CIN / 8); i += kWgThreads) {
        const int xh = i / (CIN / 8), c = i - xh * (CIN / 8);
        const int x = x0 - 1 + xh;
        const bool ok = lin && x >= 0 && x < g.X;
        cp16(su32(sIn + (size_t)(line * Xh + xh) * CIN + 8 * c),
             ok ? (const void*)(src_line + (size_t)x * CIN + 8 * c) : (const void*)a.in, ok ? 16 : 0);
      }
    }
    const bf16* gline = a.gr + ((size_t)z0 * g.Y + y0) * (size_t)g.X * COUT;
    for (int i = tid; i < g.XB * (COUT / 8); i += kWgThreads) {
      const int xo = i / (COUT / 8), c = i - xo * (COUT / 8);
      const bool ok = x0 + xo < g.X;
      cp16(su32(sG + (size_t)xo * COUT + 8 * c), ok ? (const void*)(gline + (size_t)(x0 + xo) * COUT + 8 * c)
                                                   : (const void*)a.gr,
           ok ? 16 : 0);
    }
    cp_commit_wait();
    __syncthreads();
    for (int xo = 0; xo < g.XB; ++xo) {
      float gv[COUT];
      const uint4* gs = reinterpret_cast<const uint4*>(sG + (size_t)xo * COUT);
#pragma unroll
      for (int c8 = 0; c8 < COUT / 8; ++c8) {
        const uint4 u = gs[c8];
        gv[8 * c8 + 0] = bf_lo(u.x);
        gv[8 * c8 + 1] = bf_hi(u.x);
        gv[8 * c8 + 2] = bf_lo(u.y);
        gv[8 * c8 + 3] = bf_hi(u.y);
        gv[8 * c8 + 4] = bf_lo(u.z);
        gv[8 * c8 + 5] = bf_hi(u.z);
        gv[8 * c8 + 6] = bf_lo(u.w);
        gv[8 * c8 + 7] = bf_hi(u.w);
      }
      const bf16* srow = sIn + (size_t)xo * CIN;
#pragma unroll
      for (int pp = 0; pp < PPT; ++pp) {
        const float v = __bfloat162float(srow[offs[pp]]);
#pragma unroll
        for (int c = 0; c < COUT; ++c) acc[pp][c] = fmaf(v, gv[c], acc[pp][c]);
      }
      if (tid < COUT) {
#pragma unroll
        for (int c = 0; c < COUT; ++c)
          if (c == tid) bacc += gv[c];
      }
    }
  }
  float* out = a.partial + (size_t)blockIdx.x * (NP * COUT + COUT);
#pragma unroll
  for (int pp = 0; pp < PPT; ++pp) {
    const int p = tid + pp * kWgThreads;
    if (p < NP) {
#pragma unroll
      for (int c = 0; c < COUT; ++c) out[(size_t)p * COUT + c] = acc[pp][c];
    }
  }
  if (tid < COUT) out[NP * COUT + tid] = bacc;
}

// grad[i] = sum_b partial[b][i]  (fixed order: deterministic)
__global__ void wg_reduce_kernel(const float* partial, int nparts, int n, float* grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * n + i];
  grad[i] = s;
}

// ------------------------------------------------------------ loss, Adam, packing
// dY = 2 (y - t) / (6 V) for the six output channels; loss sum of squares / (6 V)
__global__ void loss_kernel(const float* y, const float* t, bf16* dy, size_t V, double* loss) {
  __shared__ double red[256];
  const size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (v < V) {
    const float scale = 2.0f / (6.0f * (float)V);
    uint32_t pk[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) pk[c] = 0u;
#pragma unroll
    for (int c = 0; c < 6; c += 2) {
      const float d0 = y[v * 8 + c] - t[v * 8 + c];
      const float d1 = y[v * 8 + c + 1] - t[v * 8 + c + 1];
      s += (double)d0 * d0 + (double)d1 * d1;
      pk[c / 2] = pack_bf16(scale * d0, scale * d1);
    }
    uint4* dst = reinterpret_cast<uint4*>(dy + v * 16);
    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (6.0 * (double)V));
}

__global__ void adam_kernel(float* w, const float* grad, float* m, float* v, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = grad[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// forward operand of layer l: [27][CIN/8][COUT][8] from w[27][CIN][COUT];
// input-gradient operand: [27][COUT/8][CIN][8] from w[26 - tap][ci][co]
__global__ void pack_kernel(const float* params, bf16* wf, bf16* wd, int CIN, int COUT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * CIN * COUT) return;
  const int tap = i / (CIN * COUT);
  const int r = i - tap * CIN * COUT;
  const int ci = r / COUT, co = r - ci * COUT;
  const bf16 val = __float2bfloat16_rn(params[i]);
  wf[((size_t)(tap * (CIN / 8) + ci / 8) * COUT + co) * 8 + (ci & 7)] = val;
  if (wd) wd[((size_t)((26 - tap) * (COUT / 8) + co / 8) * CIN + ci) * 8 + (co & 7)] = val;
}

// ------------------------------------------------------------ features / target / apply
struct Fields {
  const float* f[6];
  int Nx, Ny, Nz, pitch;
};

__global__ void sumsq_kernel(Fields F, double* out) {
  __shared__ double red[256];
  const size_t V = (size_t)F.Nx * F.Ny * F.Nz;
  double s = 0.0;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    const size_t x = v % F.Nx, yz = v / F.Nx;
    const size_t off = yz * F.pitch + x;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double u = F.f[c][off];
      s += u * u;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

__global__ void features_kernel(Fields F, const float* ca, const float* cb, const float* cc, float tau,
                                const double* sumsq, double* s_out, bf16* X) {
  const size_t V = (size_t)F.Nx * F.Ny * F.Nz;
  const double s = sqrt(*sumsq / (6.0 * (double)V));
  const float inv = s > 0.0 ? (float)(1.0 / s) : 0.0f;
  const size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (v == 0) *s_out = s;
  if (v >= V) return;
  const size_t x = v % F.Nx, yz = v / F.Nx;
  const size_t off = yz * F.pitch + x;
  float c[16];
#pragma unroll
  for (int k = 0; k < 6; ++k) c[k] = F.f[k][off] * inv;
  c[6] = ca[off];
  c[7] = 2.0f * cb[off] / tau;
  c[8] = 4.0f * cc[off] / (tau * tau);
#pragma unroll
  for (int k = 9; k < 16; ++k) c[k] = 0.0f;
  uint4* dst = reinterpret_cast<uint4*>(X + v * 16);
  dst[0] = make_uint4(pack_bf16(c[0], c[1]), pack_bf16(c[2], c[3]), pack_bf16(c[4], c[5]), pack_bf16(c[6], c[7]));
  dst[1] = make_uint4(pack_bf16(c[8], c[9]), 0u, 0u, 0u);
}

__global__ void target_kernel(Fields fine, Fields coarse, const double* s, float* T) {
  const size_t V = (size_t)fine.Nx * fine.Ny * fine.Nz;
  const size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float inv = *s > 0.0 ? (float)(1.0 / *s) : 0.0f;
  const size_t x = v % fine.Nx, yz = v / fine.Nx;
  const size_t off = yz * fine.pitch + x;
  float o[8];
#pragma unroll
  for (int k = 0; k < 6; ++k) o[k] = (fine.f[k][off] - coarse.f[k][off]) * inv;
  o[6] = o[7] = 0.0f;
  float4* dst = reinterpret_cast<float4*>(T + v * 8);
  dst[0] = make_float4(o[0], o[1], o[2], o[3]);
  dst[1] = make_float4(o[4], o[5], o[6], o[7]);
}

// E_i is fixed on the first / last coefficient along the two axes != i, H_i
// along axis i.
struct FieldsW {
  float* f[6];
};

__global__ void apply_kernel(Fields F, FieldsW W, const double* s, const float* Y) {
  const size_t V = (size_t)F.Nx * F.Ny * F.Nz;
  const size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int x = (int)(v % F.Nx);
  const size_t yz = v / F.Nx;
  const int y = (int)(yz % F.Ny), z = (int)(yz / F.Ny);
  const bool bx = x == 0 || x == F.Nx - 1, by = y == 0 || y == F.Ny - 1, bz = z == 0 || z == F.Nz - 1;
  const bool fixed[6] = {by || bz, bx || bz, bx || by, bx, by, bz};
  const float sc = (float)*s;
  const size_t off = yz * F.pitch + x;
#pragma unroll
  for (int k = 0; k < 6; ++k)
    if (!fixed[k]) W.f[k][off] += sc * Y[v * 8 + k];
}

__global__ void distance_kernel(Fields A, Fields B, double* out) {
  __shared__ double r0[256], r1[256];
  const size_t V = (size_t)A.Nx * A.Ny * A.Nz;
  double sd = 0.0, sb = 0.0;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    const size_t x = v % A.Nx, yz = v / A.Nx;
    const size_t off = yz * A.pitch + x;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double b = B.f[c][off];
      const double d = (double)A.f[c][off] - b;
      sd += d * d;
      sb += b * b;
    }
  }
  r0[threadIdx.x] = sd;
  r1[threadIdx.x] = sb;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      r0[threadIdx.x] += r0[threadIdx.x + k];
      r1[threadIdx.x] += r1[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(out, r0[0]);
    atomicAdd(out + 1, r1[0]);
  }
}

inline unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------ the net handle
struct adi_net_ctx {
  int N[3] = {0, 0, 0};
  size_t V = 0;
  Geom g{};     // weight-gradient blocks
  Ring ring{};  // convolution work units
  void* encode = nullptr;  // cuTensorMapEncodeTiled (driver entry point)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, sms = 0;
  int optin = 0;            // opt-in shared memory per block: every convolution CTA takes all of it
  float* params = nullptr;  // master FP32 parameters
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16* wf[4] = {};  // forward operands
  bf16* wd[4] = {};  // input-gradient operands (layers 1..3)
  bf16* act[3] = {};
  bf16* dact[2] = {};
  bf16* dy = nullptr;
  float* yout = nullptr;
  float* partial = nullptr;
  double* scal = nullptr;  // [0] sum of squares, [1] s, [2] loss sum, [3..4] distance sums
  int* d_err = nullptr;
  long long adam_t = 0;
  int loss_count = 0;
  std::string err;
};

namespace {

std::string g_net_err = "no error";

adi_status net_fail(adi_net n, adi_status s, const std::string& msg) {
  if (n) n->err = msg;
  else g_net_err = msg;
  return s;
}
adi_status net_cuda(adi_net n, cudaError_t e, const char* where) {
  return net_fail(n, e == cudaErrorMemoryAllocation ? ADI_ENOMEM : ADI_ECUDA,
                  std::string(where) + ": " + cudaGetErrorString(e));
}

Fields fields_of(adi_handle h) {
  Fields F{};
  for (int k = 0; k < 6; ++k) F.f[k] = static_cast<const float*>(h->cur[k]);
  F.Nx = h->N[0];
  F.Ny = h->N[1];
  F.Nz = h->N[2];
  F.pitch = h->pitch;
  return F;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 5D view (8 channels, CIN/8 chunks, X, Y, Z) of a channels-last BF16 array; a
// box (8, 1, Xh, Yh, 1) is one chunk plane of a ring slot.  Out-of-grid voxels
// (x, y, z outside) arrive as zeros: the convolution's zero padding.
cudaError_t encode_act(adi_net n, const bf16* act, int cin, CUtensorMap* out) {
  if (((uintptr_t)act & 15u) != 0) return cudaErrorInvalidValue;
  const Ring& r = n->ring;
  cuuint64_t dims[5] = {8, (cuuint64_t)(cin / 8), (cuuint64_t)r.X, (cuuint64_t)r.Y, (cuuint64_t)r.Z};
  cuuint64_t strides[4] = {16, (cuuint64_t)cin * 2, (cuuint64_t)r.X * cin * 2, (cuuint64_t)r.X * r.Y * cin * 2};
  cuuint32_t box[5] = {8, 1, (cuuint32_t)r.Xh, (cuuint32_t)r.Yh, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult res = reinterpret_cast<EncodeTiledFn>(n->encode)(
      out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(act), dims, strides, box, estr,
      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return res == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIN, int COUT, int EPI>
cudaError_t launch_conv(adi_net n, const bf16* in, const bf16* w, const float* bias, const bf16* mask, void* out) {
  // all of the opt-in shared memory: one CTA per SM, so the 512 tensor-memory
  // columns of a CTA never wait for another CTA's
  const size_t smem = (size_t)n->optin;
  cudaError_t e = cudaFuncSetAttribute(conv_kernel<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  e = encode_act(n, in, CIN, &map);
  if (e != cudaSuccess) return e;
  ConvArgs a{w, bias, mask, out, n->ring, n->d_err};
  const int grid = n->ring.units < n->sms ? n->ring.units : n->sms;
  conv_kernel<CIN, COUT, EPI><<<grid, kConvThreads, smem, n->stream>>>(a, map);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_wgrad(adi_net n, const bf16* in, const bf16* gr, float* grad_w) {
  const int Xh = n->g.XB + 2;
  const size_t smem = (size_t)9 * Xh * CIN * 2 + (size_t)n->g.XB * COUT * 2;
  cudaError_t e = cudaFuncSetAttribute(wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  WgArgs a{in, gr, n->partial, n->g};
  const int nblk = n->g.nseg * n->g.Y * n->g.Z;
  const int grid = nblk < n->sms ? nblk : n->sms;
  wgrad_kernel<CIN, COUT><<<grid, kWgThreads, smem, n->stream>>>(a);
  const int cnt = 27 * CIN * COUT + COUT;
  wg_reduce_kernel<<<blocks_for(cnt, 256), 256, 0, n->stream>>>(n->partial, grid, cnt, grad_w);
  return cudaGetLastError();
}

cudaError_t pack_weights(adi_net n) {
  for (int l = 0; l < 4; ++l) {
    const int cnt = 27 * kCI[l] * kCO[l];
    pack_kernel<<<blocks_for(cnt, 256), 256, 0, n->stream>>>(n->params + w_off(l), n->wf[l], l > 0 ? n->wd[l] : nullptr,
                                                            kCI[l], kCO[l]);
  }
  return cudaGetLastError();
}

// forward of X into act[0..2] and the FP32 output
cudaError_t net_forward(adi_net n, const bf16* X, float* Y) {
  cudaError_t e = launch_conv<16, 32, EPI_RELU>(n, X, n->wf[0], n->params + b_off(0), nullptr, n->act[0]);
  if (e == cudaSuccess) e = launch_conv<32, 32, EPI_RELU>(n, n->act[0], n->wf[1], n->params + b_off(1), nullptr, n->act[1]);
  if (e == cudaSuccess) e = launch_conv<32, 32, EPI_RELU>(n, n->act[1], n->wf[2], n->params + b_off(2), nullptr, n->act[2]);
  if (e == cudaSuccess) e = launch_conv<32, 16, EPI_LINEAR>(n, n->act[2], n->wf[3], n->params + b_off(3), nullptr, Y);
  return e;
}

// forward + loss + backward into n->grad
cudaError_t net_backward(adi_net n, const bf16* X, const float* T) {
  cudaError_t e = net_forward(n, X, n->yout);
  if (e != cudaSuccess) return e;
  loss_kernel<<<blocks_for(n->V, 256), 256, 0, n->stream>>>(n->yout, T, n->dy, n->V, n->scal + 2);
  n->loss_count += 1;
  e = launch_wgrad<32, 16>(n, n->act[2], n->dy, n->grad + w_off(3));
  if (e == cudaSuccess) e = launch_conv<16, 32, EPI_MASK>(n, n->dy, n->wd[3], nullptr, n->act[2], n->dact[0]);
  if (e == cudaSuccess) e = launch_wgrad<32, 32>(n, n->act[1], n->dact[0], n->grad + w_off(2));
  if (e == cudaSuccess) e = launch_conv<32, 32, EPI_MASK>(n, n->dact[0], n->wd[2], nullptr, n->act[1], n->dact[1]);
  if (e == cudaSuccess) e = launch_wgrad<32, 32>(n, n->act[0], n->dact[1], n->grad + w_off(1));
  if (e == cudaSuccess) e = launch_conv<32, 32, EPI_MASK>(n, n->dact[1], n->wd[1], nullptr, n->act[0], n->dact[0]);
  if (e == cudaSuccess) e = launch_wgrad<16, 32>(n, X, n->dact[0], n->grad + w_off(0));
  return e;
}

adi_status check_handle(adi_net n, adi_handle h, const char* where) {
  if (!h) return net_fail(n, ADI_EINVAL, std::string(where) + ": NULL solver handle");
  if (h->precision != ADI_PREC_FP32) return net_fail(n, ADI_EINVAL, std::string(where) + ": the solver must be FP32");
  if (h->N[0] != n->N[0] || h->N[1] != n->N[1] || h->N[2] != n->N[2])
    return net_fail(n, ADI_EINVAL, std::string(where) + ": solver grid differs from the net's");
  return ADI_OK;
}

adi_status check_err(adi_net n, const char* where) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return net_cuda(n, e, where);
  if (err) return net_fail(n, ADI_ETIMEOUT, std::string(where) + ": a bounded device wait gave up (tensor-core MMA)");
  return ADI_OK;
}

// order work: `to` waits for everything issued so far on `from`
cudaError_t stream_wait(cudaStream_t to, cudaStream_t from) {
  if (to == from) return cudaSuccess;
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev, from);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
  cudaEventDestroy(ev);
  return e;
}

}  // namespace

extern "C" {

adi_status adi_net_create(int Nx, int Ny, int Nz, adi_net* out) {
  if (!out) return net_fail(nullptr, ADI_EINVAL, "adi_net_create: out is NULL");
  *out = nullptr;
  if (Nx < 1 || Ny < 1 || Nz < 1 || Nx > 1024)
    return net_fail(nullptr, ADI_EINVAL, "adi_net_create: grid must be >= 1 per axis and N_x <= 1024");
  adi_net n = new (std::nothrow) adi_net_ctx;
  if (!n) return net_fail(nullptr, ADI_ENOMEM, "adi_net_create: host allocation failed");
  n->N[0] = Nx;
  n->N[1] = Ny;
  n->N[2] = Nz;
  n->V = (size_t)Nx * Ny * Nz;
  n->g = make_geom(Nx, Ny, Nz);
  cudaError_t e = cudaGetDevice(&n->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, n->device);
  if (e == cudaSuccess) {
    n->ring = make_ring(Nx, Ny, Nz, n->sms);
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &n->encode, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && (q != cudaDriverEntryPointSuccess || !n->encode)) e = cudaErrorNotSupported;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) n->own_stream = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, n->stream);
  };
  const size_t P = ADI_NET_PARAMS * sizeof(float);
  alloc((void**)&n->params, P);
  alloc((void**)&n->grad, P);
  alloc((void**)&n->m, P);
  alloc((void**)&n->v, P);
  for (int l = 0; l < 4; ++l) {
    alloc((void**)&n->wf[l], 27ull * kCI[l] * kCO[l] * 2);
    if (l > 0) alloc((void**)&n->wd[l], 27ull * kCI[l] * kCO[l] * 2);
  }
  for (int k = 0; k < 3; ++k) alloc((void**)&n->act[k], n->V * 32 * 2);
  for (int k = 0; k < 2; ++k) alloc((void**)&n->dact[k], n->V * 32 * 2);
  alloc((void**)&n->dy, n->V * 16 * 2);
  alloc((void**)&n->yout, n->V * 8 * 4);
  alloc((void**)&n->partial, (size_t)(n->sms > 0 ? n->sms : 1) * (27 * 32 * 32 + 32) * 4);
  alloc((void**)&n->scal, 8 * sizeof(double));
  alloc((void**)&n->d_err, sizeof(int));
  if (e == cudaSuccess) {
    const size_t need = ring_smem<32, 32>(n->ring);
    e = cudaDeviceGetAttribute(&n->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, n->device);
    if (e == cudaSuccess && need > (size_t)n->optin) {
      adi_net_destroy(n);
      return net_fail(nullptr, ADI_EINVAL, "adi_net_create: convolution block does not fit in shared memory");
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    adi_net_destroy(n);
    return net_fail(nullptr, e == cudaErrorMemoryAllocation ? ADI_ENOMEM : ADI_ECUDA,
                    std::string("adi_net_create: ") + cudaGetErrorString(e));
  }
  *out = n;
  return ADI_OK;
}

adi_status adi_net_set_stream(adi_net n, void* stream) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_set_stream: NULL net");
  cudaError_t e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_set_stream");
  if (stream == nullptr) {
    if (!n->own_stream) {
      e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return net_cuda(n, e, "adi_net_set_stream");
      n->own_stream = true;
    }
    return ADI_OK;
  }
  if (n->own_stream) cudaStreamDestroy(n->stream);
  n->own_stream = false;
  n->stream = (cudaStream_t)stream;
  return ADI_OK;
}

adi_status adi_net_set_params(adi_net n, const float* w, size_t count) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_set_params: NULL net");
  if (!w || count != (size_t)ADI_NET_PARAMS)
    return net_fail(n, ADI_EINVAL, "adi_net_set_params: w must hold ADI_NET_PARAMS floats");
  for (size_t i = 0; i < count; ++i)
    if (!std::isfinite(w[i])) return net_fail(n, ADI_ENUMERIC, "adi_net_set_params: NaN or Inf in w");
  const size_t P = count * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(n->params, w, P, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, P, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, P, n->stream);
  if (e == cudaSuccess) e = pack_weights(n);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_set_params");
  n->adam_t = 0;
  return ADI_OK;
}

adi_status adi_net_get_params(adi_net n, float* w, size_t count) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_get_params: NULL net");
  if (!w || count != (size_t)ADI_NET_PARAMS)
    return net_fail(n, ADI_EINVAL, "adi_net_get_params: w must hold ADI_NET_PARAMS floats");
  cudaError_t e = cudaMemcpyAsync(w, n->params, count * sizeof(float), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_get_params");
  return ADI_OK;
}

adi_status adi_net_features(adi_net n, adi_handle h, void* X) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_features: NULL net");
  adi_status s = check_handle(n, h, "adi_net_features");
  if (s != ADI_OK) return s;
  if (!X) return net_fail(n, ADI_EINVAL, "adi_net_features: X is NULL");
  if (!h->factored) return net_fail(n, ADI_ESTATE, "adi_net_features: the solver is not factored");
  const Fields F = fields_of(h);
  cudaError_t e = stream_wait(n->stream, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->scal, 0, sizeof(double), n->stream);
  if (e == cudaSuccess) {
    sumsq_kernel<<<2 * n->sms, 256, 0, n->stream>>>(F, n->scal);
    features_kernel<<<blocks_for(n->V, 256), 256, 0, n->stream>>>(
        F, static_cast<const float*>(h->coef[0]), static_cast<const float*>(h->coef[1]),
        static_cast<const float*>(h->coef[2]), (float)h->dt, n->scal, n->scal + 1, static_cast<bf16*>(X));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_features");
  return ADI_OK;
}

adi_status adi_net_target(adi_net n, adi_handle fine, adi_handle coarse, float* T) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_target: NULL net");
  adi_status s = check_handle(n, fine, "adi_net_target");
  if (s == ADI_OK) s = check_handle(n, coarse, "adi_net_target");
  if (s != ADI_OK) return s;
  if (!T) return net_fail(n, ADI_EINVAL, "adi_net_target: T is NULL");
  cudaError_t e = stream_wait(n->stream, fine->stream);
  if (e == cudaSuccess) e = stream_wait(n->stream, coarse->stream);
  if (e == cudaSuccess) {
    target_kernel<<<blocks_for(n->V, 256), 256, 0, n->stream>>>(fields_of(fine), fields_of(coarse), n->scal + 1, T);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_target");
  return ADI_OK;
}

adi_status adi_net_forward(adi_net n, const void* X, float* Y) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_forward: NULL net");
  if (!X || !Y) return net_fail(n, ADI_EINVAL, "adi_net_forward: NULL array");
  if (((uintptr_t)X & 15u) || ((uintptr_t)Y & 15u))
    return net_fail(n, ADI_EINVAL, "adi_net_forward: X and Y must be 16-byte aligned");
  cudaError_t e = net_forward(n, static_cast<const bf16*>(X), Y);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_forward");
  return ADI_OK;
}

adi_status adi_net_apply(adi_net n, adi_handle h, const float* Y) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_apply: NULL net");
  adi_status s = check_handle(n, h, "adi_net_apply");
  if (s != ADI_OK) return s;
  if (!Y) return net_fail(n, ADI_EINVAL, "adi_net_apply: Y is NULL");
  FieldsW W;
  for (int k = 0; k < 6; ++k) W.f[k] = static_cast<float*>(h->cur[k]);
  cudaError_t e = stream_wait(n->stream, h->stream);
  if (e == cudaSuccess) {
    apply_kernel<<<blocks_for(n->V, 256), 256, 0, n->stream>>>(fields_of(h), W, n->scal + 1, Y);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = stream_wait(h->stream, n->stream);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_apply");
  return ADI_OK;
}

adi_status adi_net_train_step(adi_net n, const void* X, const float* T, float lr) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_train_step: NULL net");
  if (!X || !T) return net_fail(n, ADI_EINVAL, "adi_net_train_step: NULL array");
  if (((uintptr_t)X & 15u) || ((uintptr_t)T & 15u))
    return net_fail(n, ADI_EINVAL, "adi_net_train_step: X and T must be 16-byte aligned");
  if (!(lr > 0.0f) || !std::isfinite(lr)) return net_fail(n, ADI_EINVAL, "adi_net_train_step: lr must be > 0");
  cudaError_t e = net_backward(n, static_cast<const bf16*>(X), T);
  if (e == cudaSuccess) {
    n->adam_t += 1;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)n->adam_t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)n->adam_t));
    adam_kernel<<<blocks_for(ADI_NET_PARAMS, 256), 256, 0, n->stream>>>(n->params, n->grad, n->m, n->v,
                                                                        ADI_NET_PARAMS, lr, c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = pack_weights(n);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_train_step");
  return ADI_OK;
}

adi_status adi_net_gradient(adi_net n, const void* X, const float* T, float* grad, double* loss) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_gradient: NULL net");
  if (!X || !T || !grad || !loss) return net_fail(n, ADI_EINVAL, "adi_net_gradient: NULL argument");
  cudaError_t e = cudaMemsetAsync(n->scal + 2, 0, sizeof(double), n->stream);
  if (e == cudaSuccess) e = net_backward(n, static_cast<const bf16*>(X), T);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(grad, n->grad, ADI_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss, n->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->scal + 2, 0, sizeof(double), n->stream);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_gradient");
  n->loss_count = 0;
  return check_err(n, "adi_net_gradient");
}

adi_status adi_net_loss(adi_net n, double* sum, int* count) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_net_loss: NULL net");
  if (!sum || !count) return net_fail(n, ADI_EINVAL, "adi_net_loss: NULL argument");
  cudaError_t e = cudaMemcpyAsync(sum, n->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->scal + 2, 0, sizeof(double), n->stream);
  if (e != cudaSuccess) return net_cuda(n, e, "adi_net_loss");
  adi_status s = check_err(n, "adi_net_loss");
  *count = n->loss_count;
  n->loss_count = 0;
  return s;
}

adi_status adi_fields_distance(adi_handle a, adi_handle b, double* rel) {
  if (!a || !b || !rel) return net_fail(nullptr, ADI_EINVAL, "adi_fields_distance: NULL argument");
  if (a->precision != ADI_PREC_FP32 || b->precision != ADI_PREC_FP32)
    return net_fail(nullptr, ADI_EINVAL, "adi_fields_distance: both solvers must be FP32");
  if (a->N[0] != b->N[0] || a->N[1] != b->N[1] || a->N[2] != b->N[2])
    return net_fail(nullptr, ADI_EINVAL, "adi_fields_distance: grids differ");
  double* d = nullptr;
  double hsum[2] = {0.0, 0.0};
  cudaError_t e = stream_wait(a->stream, b->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&d, 2 * sizeof(double), a->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, 2 * sizeof(double), a->stream);
  if (e == cudaSuccess) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device);
    distance_kernel<<<2 * (sms > 0 ? sms : 1), 256, 0, a->stream>>>(fields_of(a), fields_of(b), d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hsum, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, a->stream);
  if (d) cudaFreeAsync(d, a->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
  if (e != cudaSuccess)
    return net_fail(nullptr, ADI_ECUDA, std::string("adi_fields_distance: ") + cudaGetErrorString(e));
  *rel = hsum[1] > 0.0 ? std::sqrt(hsum[0] / hsum[1]) : std::sqrt(hsum[0]);
  return ADI_OK;
}

adi_status adi_copy_state(adi_handle dst, adi_handle src) {
  if (!dst || !src) return net_fail(nullptr, ADI_EINVAL, "adi_copy_state: NULL handle");
  if (dst->N[0] != src->N[0] || dst->N[1] != src->N[1] || dst->N[2] != src->N[2] || dst->p != src->p ||
      dst->precision != src->precision)
    return net_fail(nullptr, ADI_EINVAL, "adi_copy_state: grids, degrees or precisions differ");
  cudaError_t e = cudaStreamSynchronize(src->stream);
  const double t = src->t_host + (double)src->steps_host * src->dt;
  for (int k = 0; k < 6 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(dst->cur[k], src->cur[k], dst->Np * dst->esize, cudaMemcpyDeviceToDevice, dst->stream);
  if (e == cudaSuccess) e = adi::set_clock(*dst, t);
  if (e != cudaSuccess) return net_fail(nullptr, ADI_ECUDA, std::string("adi_copy_state: ") + cudaGetErrorString(e));
  dst->t_host = t;
  dst->steps_host = 0;
  return ADI_OK;
}

adi_status adi_corrector_run(adi_net n, adi_handle coarse, adi_handle fine, int m, int k, int guard_every, double tol,
                             int* n_fallback, double* max_err) {
  if (!n) return net_fail(nullptr, ADI_EINVAL, "adi_corrector_run: NULL net");
  adi_status s = check_handle(n, coarse, "adi_corrector_run");
  if (s == ADI_OK) s = check_handle(n, fine, "adi_corrector_run");
  if (s != ADI_OK) return s;
  if (m < 1 || k < 1 || guard_every < 1 || !(tol > 0.0) || !n_fallback || !max_err)
    return net_fail(n, ADI_EINVAL, "adi_corrector_run: need m, k, guard_every >= 1, tol > 0 and output pointers");
  if (std::fabs(coarse->dt - k * fine->dt) > 1e-12 * coarse->dt)
    return net_fail(n, ADI_EINVAL, "adi_corrector_run: coarse dt must be k times fine dt");
  *n_fallback = 0;
  *max_err = 0.0;
  bf16* X = nullptr;
  float* Y = nullptr;
  cudaError_t e = cudaMalloc((void**)&X, n->V * 16 * 2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&Y, n->V * 8 * 4);
  if (e != cudaSuccess) {
    cudaFree(X);
    return net_cuda(n, e, "adi_corrector_run");
  }
  auto corrected_step = [&]() -> adi_status {
    adi_status r = adi_step(coarse, 1);
    if (r == ADI_OK) r = adi_net_features(n, coarse, X);
    if (r == ADI_OK) r = adi_net_forward(n, X, Y);
    if (r == ADI_OK) r = adi_net_apply(n, coarse, Y);
    return r;
  };
  adi_status r = ADI_OK;
  for (int done = 0; done < m && r == ADI_OK;) {
    const int win = (m - done) < guard_every ? (m - done) : guard_every;
    // guard: the window's first step both ways
    r = adi_copy_state(fine, coarse);
    if (r == ADI_OK) r = adi_step(fine, k);
    if (r == ADI_OK) r = corrected_step();
    double d = 0.0;
    if (r == ADI_OK) r = adi_fields_distance(coarse, fine, &d);
    if (r != ADI_OK) break;
    if (d > *max_err) *max_err = d;
    if (!(d <= tol)) {
      *n_fallback += 1;
      if (win > 1) r = adi_step(fine, k * (win - 1));
      if (r == ADI_OK) r = adi_copy_state(coarse, fine);
    } else {
      for (int i = 1; i < win && r == ADI_OK; ++i) r = corrected_step();
    }
    done += win;
  }
  if (r == ADI_OK) {
    e = cudaStreamSynchronize(coarse->stream);
    if (e != cudaSuccess) r = net_cuda(n, e, "adi_corrector_run");
  }
  cudaFree(X);
  cudaFree(Y);
  if (r != ADI_OK && n->err.empty()) n->err = "adi_corrector_run: a solver call failed";
  if (r == ADI_OK) r = check_err(n, "adi_corrector_run");
  return r;
}

void adi_net_destroy(adi_net n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  cudaFree(n->params);
  cudaFree(n->grad);
  cudaFree(n->m);
  cudaFree(n->v);
  for (int l = 0; l < 4; ++l) {
    cudaFree(n->wf[l]);
    cudaFree(n->wd[l]);
  }
  for (int k = 0; k < 3; ++k) cudaFree(n->act[k]);
  for (int k = 0; k < 2; ++k) cudaFree(n->dact[k]);
  cudaFree(n->dy);
  cudaFree(n->yout);
  cudaFree(n->partial);
  cudaFree(n->scal);
  cudaFree(n->d_err);
  if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
  delete n;
}

const char* adi_net_last_error(adi_net n) { return n ? n->err.c_str() : g_net_err.c_str(); }

}  // extern "C"
