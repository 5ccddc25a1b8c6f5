// unet_conv.cu -- tensor-core (tcgen05) kernels of the U-Net warm start:
// the 3x3x3 convolution as an implicit GEMM (forward, and data gradient with
// the flipped, transposed weight image) and the weight gradient.
//
// Convolution, one CTA of 128 threads per T tiles of 128 consecutive voxel rows:
//   D[row][co] = sum over 3 dz planes x (cin / 16) channel chunks x 9 (dy, dx)
//   taps of A_tap[row][16 ci] x B_tap[co][16 ci], with A_tap the input rows
//   shifted by the tap (padded layout, see unet_internal.cuh).
//   Per (dz, chunk) stage one bulk copy brings a slab of 128 T + 2 Wp + 2 input
//   rows per 8-channel block into shared memory (K-major no-swizzle operand:
//   core matrices of 8 rows x 16 bytes, rows 16 bytes apart), so the nine
//   (dy, dx) taps of all T tiles are descriptor start offsets into one slab;
//   another brings the stage's pre-arranged weight image (K-major, N = cout).
//   Warp 0 lane 0 issues the copies, warp 1 lane 0 the MMAs (M = 128,
//   N = cout, K = 16, FP32 accumulators in TMEM: T x cout columns), and all four
//   warps then read the accumulators (tcgen05.ld, lane = row) and write the
//   interior rows as BF16 with the optional ReLU or ReLU-mask of the backward
//   pass. Stages are double/triple buffered on full/empty mbarriers.
// Weight gradient: dw[tap][co][ci] = sum_r in[r + off(tap)][ci] dz[r][co], an
//   MMA with M = 128 input channels (one tile of 16 channel blocks; rows past
//   the tensor's channels are computed and dropped), N = cout and K = voxel rows,
//   both operands MN-major (channels contiguous in a 16-byte row). CTAs stride
//   over chunks of K rows, accumulate 9 or 3 taps in TMEM, and add their sums to
//   the FP32 gradient with atomics.
// Every mbarrier wait is bounded (2 s); a wait that runs out sets an error bit,
// the CTA drains the copies it issued, frees its TMEM and returns.
#include <algorithm>
#include <cstdio>

#include "tc_ptx.cuh"
#include "unet_internal.cuh"

namespace unet {

constexpr uint64_t kWaitNs = 2000000000ull;
static unsigned long long g_launches = 0;
uint64_t launch_count() { return g_launches; }

__device__ __forceinline__ bool row_interior(const Vol& v, long long r) {
  if (r >= v.r_end) return false;
  const long long z = r / v.P;
  const long long rem = r - z * v.P;
  const int y = (int)(rem / v.Wp);
  const int x = (int)(rem - (long long)y * v.Wp);
  return z >= 1 && z <= v.D && y >= 1 && y <= v.H && x >= 1 && x <= v.W;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ bool bf16_positive(uint32_t bits16) { return (int16_t)(bits16 & 0xFFFFu) > 0; }

// ---------------------------------------------------------------------------
// 3x3x3 convolution
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kConvThreads, 1) k_conv3(const __grid_constant__ ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)a.nstage * a.stage_bytes);
  uint64_t* empty = full + kMaxStages;
  uint64_t* done = empty + kMaxStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* consumed = abort_flag + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = a.v.r_begin + (long long)blockIdx.x * 128 * a.T;
  const int nst = 3 * a.nchunk;
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nstage; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    *consumed = 0;
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  int issued = 0;
  if (warp == 0 && lane == 0) {
    // producer: one input slab (two 8-channel blocks) and one weight image per stage
    for (int s = 0; s < nst; ++s) {
      const int b = s % a.nstage;
      if (s >= a.nstage && !tc::mbar_wait(&empty[b], ((s / a.nstage) - 1) & 1, kWaitNs)) {
        atomicOr(a.err, kErrWaitProducer);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const int dz = s / a.nchunk, c = s - dz * a.nchunk;
      uint8_t* A = smem + (size_t)b * a.stage_bytes;
      uint8_t* B = A + a.a_bytes;
      tc::mbar_arrive_expect_tx(&full[b], a.a_bytes + a.b_bytes);
      const __nv_bfloat16* src = c < a.nchunk0 ? a.src0 : a.src1;
      const long long g0 = 2ll * (c < a.nchunk0 ? c : c - a.nchunk0);
      const long long start = r0 + (long long)(dz - 1) * a.v.P - a.v.Wp - 1;
      tc::bulk_g2s(A, src + (g0 * a.v.rows + start) * 8, (uint32_t)a.R * 16u, &full[b]);
      tc::bulk_g2s(A + (size_t)a.R * 16, src + ((g0 + 1) * a.v.rows + start) * 8, (uint32_t)a.R * 16u, &full[b]);
      tc::bulk_g2s(B, a.wimg + (size_t)s * (a.b_bytes / 2), a.b_bytes, &full[b]);
      issued = s + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = tc::idesc_bf16(128, a.cout, 0, 0);
    const uint32_t lbo_a = (uint32_t)a.R * 16u, lbo_b = (uint32_t)a.cout * 16u;
    int s = 0;
    for (; s < nst; ++s) {
      const int b = s % a.nstage;
      if (!tc::mbar_wait(&full[b], (s / a.nstage) & 1, kWaitNs)) {
        atomicOr(a.err, kErrWaitMma);
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t A = tc::smem_u32(smem + (size_t)b * a.stage_bytes);
      const uint32_t B = A + a.a_bytes;
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap - 3 * dy;
        const uint64_t bd = tc::sdesc(B + (uint32_t)tap * 2u * lbo_b, lbo_b, 128);
        const uint32_t shift = (uint32_t)(dy * a.v.Wp + dx) * 16u;
        for (int t = 0; t < a.T; ++t) {
          const uint64_t ad = tc::sdesc(A + shift + (uint32_t)t * 2048u, lbo_a, 128);
          tc::mma_bf16(tmem + (uint32_t)(t * a.cout), ad, bd, idesc, (s | tap) != 0 ? 1u : 0u);
        }
      }
      tc::mma_commit(&empty[b]);
    }
    *consumed = s;
    tc::mma_commit(done);
  }
  __syncwarp();

  // epilogue: TMEM lane = row of the tile
  const bool ok = tc::mbar_wait(done, 0, kWaitNs);
  if (!ok) atomicOr(a.err, kErrWaitDone);
  tc::fence_after_sync();
  const int good = __syncthreads_and(ok && !*abort_flag);
  if (good) {
    const int m = warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int t = 0; t < a.T; ++t) {
      const long long r = r0 + (long long)t * 128 + m;
      const bool inside = row_interior(a.v, r);
      for (int c0 = 0; c0 < a.cout; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + lane_base + (uint32_t)(t * a.cout + c0), v);
        if (!inside) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int gidx = (c0 >> 3) + half;
          const bool first = gidx < a.dgroups0;
          const long long gl = first ? gidx : gidx - a.dgroups0;
          float* f = v + 8 * half;
          if (a.relu) {
#pragma unroll
            for (int j = 0; j < 8; ++j) f[j] = fmaxf(f[j], 0.f);
          }
          const __nv_bfloat16* mk = first ? a.mask0 : a.mask1;
          if (mk) {
            const uint4 mv = *reinterpret_cast<const uint4*>(mk + (gl * a.v.rows + r) * 8);
            const uint32_t w4[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (!bf16_positive(w4[j])) f[2 * j] = 0.f;
              if (!bf16_positive(w4[j] >> 16)) f[2 * j + 1] = 0.f;
            }
          }
          uint4 o;
          o.x = pack2(f[0], f[1]);
          o.y = pack2(f[2], f[3]);
          o.z = pack2(f[4], f[5]);
          o.w = pack2(f[6], f[7]);
          __nv_bfloat16* d = first ? a.dst0 : a.dst1;
          *reinterpret_cast<uint4*>(d + (gl * a.v.rows + r) * 8) = o;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    // copies issued but never consumed (only after a wait ran out) land before the CTA leaves
    for (int s = *consumed; s < issued; ++s) tc::mbar_wait(&full[s % a.nstage], (s / a.nstage) & 1, kWaitNs);
    if (!ok) tc::mbar_wait(done, 0, kWaitNs);
  }
  __syncwarp();
  if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

// ---------------------------------------------------------------------------
// 3x3x3 convolution, input planes streamed through a column of output planes
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kConvThreads, 1) k_conv3z(const __grid_constant__ ConvZArgs z) {
  const ConvArgs& a = z.c;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + z.a_region + 2 * (size_t)z.bz_bytes);
  uint64_t* empty = full + kMaxStages;
  uint64_t* done = empty + kMaxStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* consumed = abort_flag + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long u0 = z.u_begin + (long long)blockIdx.x * 128 * a.T;
  const int z0 = 1 + blockIdx.y * z.Zc;                 // first output plane
  const int p_last = min(z0 + z.Zc, a.v.D + 1);         // last input plane streamed (halo plane at most)
  const int np = p_last - (z0 - 1) + 1;                 // input planes
  const int nst = a.nchunk * np;                        // stages: chunk-major, planes inner
  const int cout = a.cout;
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nstage; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    *consumed = 0;
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  {  // every accumulator starts at zero: each MMA below accumulates
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (uint32_t c0 = 0; c0 < a.tmem_cols; c0 += 16) tc::tmem_zero16(tmem + lane_base + c0);
    tc::tmem_wait_st();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  int issued = 0;
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < nst; ++s) {
      const int b = s % a.nstage;
      if (s >= a.nstage && !tc::mbar_wait(&empty[b], ((s / a.nstage) - 1) & 1, kWaitNs)) {
        atomicOr(a.err, kErrWaitProducer);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const int c = s / np, i = s - c * np;
      const int p = z0 - 1 + i;
      uint8_t* A = smem + (size_t)b * a.a_bytes;
      const bool loadB = i == 0;  // chunk c's image, into buffer c & 1 (free: see below)
      tc::mbar_arrive_expect_tx(&full[b], a.a_bytes + (loadB ? z.bz_bytes : 0u));
      const __nv_bfloat16* src = c < a.nchunk0 ? a.src0 : a.src1;
      const long long g0 = 2ll * (c < a.nchunk0 ? c : c - a.nchunk0);
      const long long start = (long long)p * a.v.P + u0 - a.v.Wp - 1;
      tc::bulk_g2s(A, src + (g0 * a.v.rows + start) * 8, (uint32_t)a.R * 16u, &full[b]);
      tc::bulk_g2s(A + (size_t)a.R * 16, src + ((g0 + 1) * a.v.rows + start) * 8, (uint32_t)a.R * 16u, &full[b]);
      // The image buffer c & 1 was last read by chunk c - 2, whose stages end at
      // s - np - 1 <= s - nstage: the empty wait above covered them.
      if (loadB)
        tc::bulk_g2s(smem + z.a_region + (size_t)(c & 1) * z.bz_bytes, z.zimg + (size_t)c * (z.bz_bytes / 2),
                     z.bz_bytes, &full[b]);
      issued = s + 1;
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t lbo_a = (uint32_t)a.R * 16u, lbo_b = 3u * (uint32_t)cout * 16u;
    int s = 0;
    for (; s < nst; ++s) {
      const int b = s % a.nstage;
      if (!tc::mbar_wait(&full[b], (s / a.nstage) & 1, kWaitNs)) {
        atomicOr(a.err, kErrWaitMma);
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      const int c = s / np, i = s - c * np;
      const int p = z0 - 1 + i;
      // output planes q = p + 1 - k for dz taps k in [k_lo, k_hi] that land in [z0, z0 + Zc - 1]
      const int k_lo = max(0, p + 1 - (z0 + z.Zc - 1)), k_hi = min(2, p + 1 - z0);
      if (k_hi >= k_lo) {
        const int nk = k_hi - k_lo + 1;
        const uint32_t idesc = tc::idesc_bf16(128, nk * cout, 0, 0);
        const uint32_t A = tc::smem_u32(smem + (size_t)b * a.a_bytes);
        const uint32_t B = tc::smem_u32(smem + z.a_region + (size_t)(c & 1) * z.bz_bytes) +
                           (uint32_t)(k_lo * cout) * 16u;
        const int slot = z0 + z.Zc - 1 - (p + 1 - k_lo);  // TMEM block of plane p + 1 - k_lo
        // the descriptors' address field is (address >> 4): offsets add to it directly
        const uint64_t ad0 = tc::sdesc(A, lbo_a, 128), bd0 = tc::sdesc(B, lbo_b, 128);
        const uint32_t dstep = (uint32_t)(z.Zc * cout);
        const uint32_t d0 = tmem + (uint32_t)(slot * cout);
#pragma unroll 1
        for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const uint64_t bd = bd0 + (uint64_t)((uint32_t)(dy * 3 + dx) * 2u * (lbo_b >> 4));
            const uint64_t ad = ad0 + (uint64_t)(uint32_t)(dy * a.v.Wp + dx);
            for (int t = 0; t < a.T; ++t) tc::mma_bf16(d0 + (uint32_t)t * dstep, ad + (uint64_t)(t * 128), bd, idesc, 1u);
          }
        }
      }
      tc::mma_commit(&empty[b]);
    }
    *consumed = s;
    tc::mma_commit(done);
  }
  __syncwarp();

  const bool ok = tc::mbar_wait(done, 0, kWaitNs);
  if (!ok) atomicOr(a.err, kErrWaitDone);
  tc::fence_after_sync();
  const int good = __syncthreads_and(ok && !*abort_flag);
  if (good) {
    const int m = warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int t = 0; t < a.T; ++t) {
      const long long u = u0 + (long long)t * 128 + m;
      bool inplane = u < z.u_end;
      if (inplane) {
        const int uu = (int)u;  // in-plane rows fit 32 bits
        const int y = uu / a.v.Wp, x = uu - y * a.v.Wp;
        inplane = y >= 1 && y <= a.v.H && x >= 1 && x <= a.v.W;
      }
      if (cout == 16 && (z.Zc & 3) == 0 && !a.mask0 && !a.mask1 && a.dgroups0 == 2) {
        // four planes per TMEM read (64 columns), ReLU, two 16-byte rows each
        for (int s4 = 0; s4 < z.Zc; s4 += 4) {
          float v[64];
          tc::tmem_ld64(tmem + lane_base + (uint32_t)((t * z.Zc + s4) * 16), v);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int q = z0 + z.Zc - 1 - (s4 + k);
            if (!inplane || q > a.v.D) continue;
            const long long r = (long long)q * a.v.P + u;
            float* f = v + 16 * k;
            if (a.relu) {
#pragma unroll
              for (int j = 0; j < 16; ++j) f[j] = fmaxf(f[j], 0.f);
            }
            uint4 o0, o1;
            o0.x = pack2(f[0], f[1]);
            o0.y = pack2(f[2], f[3]);
            o0.z = pack2(f[4], f[5]);
            o0.w = pack2(f[6], f[7]);
            o1.x = pack2(f[8], f[9]);
            o1.y = pack2(f[10], f[11]);
            o1.z = pack2(f[12], f[13]);
            o1.w = pack2(f[14], f[15]);
            *reinterpret_cast<uint4*>(a.dst0 + r * 8) = o0;
            *reinterpret_cast<uint4*>(a.dst0 + (a.v.rows + r) * 8) = o1;
          }
        }
        continue;
      }
      for (int slot = 0; slot < z.Zc; ++slot) {
        const int q = z0 + z.Zc - 1 - slot;
        const bool inside = inplane && q <= a.v.D;
        const long long r = (long long)q * a.v.P + u;
        for (int c0 = 0; c0 < cout; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tmem + lane_base + (uint32_t)((t * z.Zc + slot) * cout + c0), v);
          if (!inside) continue;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int gidx = (c0 >> 3) + half;
            const bool first = gidx < a.dgroups0;
            const long long gl = first ? gidx : gidx - a.dgroups0;
            float* f = v + 8 * half;
            if (a.relu) {
#pragma unroll
              for (int j = 0; j < 8; ++j) f[j] = fmaxf(f[j], 0.f);
            }
            const __nv_bfloat16* mk = first ? a.mask0 : a.mask1;
            if (mk) {
              const uint4 mv = *reinterpret_cast<const uint4*>(mk + (gl * a.v.rows + r) * 8);
              const uint32_t w4[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (!bf16_positive(w4[j])) f[2 * j] = 0.f;
                if (!bf16_positive(w4[j] >> 16)) f[2 * j + 1] = 0.f;
              }
            }
            uint4 o;
            o.x = pack2(f[0], f[1]);
            o.y = pack2(f[2], f[3]);
            o.z = pack2(f[4], f[5]);
            o.w = pack2(f[6], f[7]);
            __nv_bfloat16* d = first ? a.dst0 : a.dst1;
            *reinterpret_cast<uint4*>(d + (gl * a.v.rows + r) * 8) = o;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = *consumed; s < issued; ++s) tc::mbar_wait(&full[s % a.nstage], (s / a.nstage) & 1, kWaitNs);
    if (!ok) tc::mbar_wait(done, 0, kWaitNs);
  }
  __syncwarp();
  if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

// ---------------------------------------------------------------------------
// weight gradient
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kConvThreads, 1) k_wgrad(const __grid_constant__ WgradArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.smem_main);
  uint64_t* empty = full + kMaxStages;
  uint64_t* done = empty + kMaxStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* consumed = abort_flag + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g_lo = blockIdx.z * 16;
  const int ng = min(16, a.gin - g_lo);
  int dz, dy0, ndy;
  if (a.taps == 9) {
    dz = blockIdx.y;
    dy0 = 0;
    ndy = 3;
  } else {
    dz = blockIdx.y / 3;
    dy0 = blockIdx.y - 3 * dz;
    ndy = 1;
  }
  const long long nmine = ((long long)blockIdx.x < a.nchunks)
                              ? (a.nchunks - 1 - (long long)blockIdx.x) / gridDim.x + 1
                              : 0;
  const int gout = a.cout / 8;
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nstage; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    *consumed = 0;
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  long long issued = 0;
  if (nmine > 0 && warp == 0 && lane == 0) {
    for (long long i = 0; i < nmine; ++i) {
      const int b = (int)(i % a.nstage);
      if (i >= a.nstage && !tc::mbar_wait(&empty[b], (uint32_t)((i / a.nstage) - 1) & 1u, kWaitNs)) {
        atomicOr(a.err, kErrWaitProducer);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const long long p0 = a.v.r_begin + ((long long)blockIdx.x + i * gridDim.x) * a.Kc;
      uint8_t* X = smem + (size_t)b * a.x_bytes;
      uint8_t* Z = smem + a.x_region + (size_t)b * a.dz_bytes;
      tc::mbar_arrive_expect_tx(&full[b], (uint32_t)ng * a.R * 16u + a.dz_bytes);
      const long long start = p0 + (long long)(dz - 1) * a.v.P - a.v.Wp - 1;
      for (int g = 0; g < ng; ++g) {
        const int gg = g_lo + g;
        const __nv_bfloat16* src = gg < a.gin0 ? a.src0 + (long long)gg * a.v.rows * 8
                                                : a.src1 + (long long)(gg - a.gin0) * a.v.rows * 8;
        tc::bulk_g2s(X + (size_t)g * a.R * 16, src + start * 8, (uint32_t)a.R * 16u, &full[b]);
      }
      for (int g = 0; g < gout; ++g)
        tc::bulk_g2s(Z + (size_t)g * a.Kc * 16, a.dz + ((long long)g * a.v.rows + p0) * 8, (uint32_t)a.Kc * 16u,
                     &full[b]);
      issued = i + 1;
    }
  } else if (nmine > 0 && warp == 1 && lane == 0) {
    const uint32_t idesc = tc::idesc_bf16(128, a.cout, 1, 1);
    const uint32_t sbo_a = (uint32_t)a.R * 16u, sbo_b = (uint32_t)a.Kc * 16u;
    long long i = 0;
    for (; i < nmine; ++i) {
      const int b = (int)(i % a.nstage);
      if (!tc::mbar_wait(&full[b], (uint32_t)(i / a.nstage) & 1u, kWaitNs)) {
        atomicOr(a.err, kErrWaitMma);
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t X = tc::smem_u32(smem + (size_t)b * a.x_bytes);
      const uint32_t Z = tc::smem_u32(smem + a.x_region + (size_t)b * a.dz_bytes);
      for (int ti = 0; ti < a.taps; ++ti) {
        const int dy = dy0 + ti / 3, dx = ti - 3 * (ti / 3);
        const uint32_t shift = (uint32_t)(dy * a.v.Wp + dx) * 16u;
        for (int ks = 0; ks < a.Kc / 16; ++ks) {
          const uint64_t ad = tc::sdesc(X + shift + (uint32_t)ks * 256u, 128, sbo_a);
          const uint64_t bd = tc::sdesc(Z + (uint32_t)ks * 256u, 128, sbo_b);
          tc::mma_bf16(tmem + (uint32_t)(ti * a.cout), ad, bd, idesc, (i | (long long)ks) != 0 ? 1u : 0u);
        }
      }
      tc::mma_commit(&empty[b]);
    }
    *consumed = (int)i;
    tc::mma_commit(done);
  } else if (nmine == 0 && threadIdx.x == 0) {
    tc::mbar_arrive(done);  // nothing to accumulate
  }
  __syncwarp();
  const bool ok = tc::mbar_wait(done, 0, kWaitNs);
  if (!ok) atomicOr(a.err, kErrWaitDone);
  tc::fence_after_sync();
  const int good = __syncthreads_and(ok && !*abort_flag && nmine > 0);
  if (good) {
    const int m = warp * 32 + lane;
    const bool valid = m < ng * 8;
    const int ci = g_lo * 8 + m;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int ti = 0; ti < a.taps; ++ti) {
      const int dy = dy0 + ti / 3, dx = ti - 3 * (ti / 3);
      const int tap = dz * 9 + dy * 3 + dx;
      for (int c0 = 0; c0 < a.cout; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + lane_base + (uint32_t)(ti * a.cout + c0), v);
        if (!valid) continue;
        float* base = a.dw + ((size_t)tap * a.cout + c0) * a.cin + ci;
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(base + (size_t)j * a.cin, v[j]);
      }
    }
  }
  (void)ndy;
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (long long s = *consumed; s < issued; ++s)
      tc::mbar_wait(&full[s % a.nstage], (uint32_t)(s / a.nstage) & 1u, kWaitNs);
    if (!ok) tc::mbar_wait(done, 0, kWaitNs);
  }
  __syncwarp();
  if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
constexpr int kSmemMax = 227 * 1024;
constexpr int kSmemPerSM = 228 * 1024;

// Dynamic shared memory of a CTA that holds tmem_cols TMEM columns: at least
// enough that no more CTAs share an SM than its 512 columns hold, so a
// tcgen05.alloc never waits for another CTA's columns.
static size_t smem_floor(size_t need, uint32_t tmem_cols) {
  const size_t fit = 512 / (tmem_cols ? tmem_cols : 512);
  const size_t floor_b = kSmemPerSM / (fit + 1) + 1024;
  return need > floor_b ? need : floor_b;
}

void launch_conv3(const ConvArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv3, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    attr = true;
  }
  const long long rows = a.v.r_end - a.v.r_begin;
  const long long grid = (rows + 128ll * a.T - 1) / (128ll * a.T);
  const size_t smem = smem_floor((size_t)a.nstage * a.stage_bytes + 256, a.tmem_cols);
  ++g_launches;
  k_conv3<<<(unsigned)grid, kConvThreads, smem, s>>>(a);
}

void launch_conv3z(const ConvZArgs& z, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv3z, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    attr = true;
  }
  const long long rows = z.u_end - z.u_begin;
  const long long gx = (rows + 128ll * z.c.T - 1) / (128ll * z.c.T);
  const int gy = (z.c.v.D + z.Zc - 1) / z.Zc;
  const size_t smem = smem_floor((size_t)z.a_region + 2 * (size_t)z.bz_bytes + 256, z.c.tmem_cols);
  ++g_launches;
  k_conv3z<<<dim3((unsigned)gx, gy), kConvThreads, smem, s>>>(z);
}

void launch_wgrad(const WgradArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    attr = true;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  const int gy = a.taps == 9 ? 3 : 9;
  const int gz = (a.gin + 15) / 16;
  long long gx = (2ll * sms + gy * gz - 1) / (gy * gz);
  gx = std::max(1ll, std::min(gx, a.nchunks));
  const size_t smem = smem_floor((size_t)a.smem_main + 256, a.tmem_cols);
  ++g_launches;
  k_wgrad<<<dim3((unsigned)gx, gy, gz), kConvThreads, smem, s>>>(a);
}

}  // namespace unet
