// unet_internal.cuh -- data layout and kernel arguments of the U-Net warm start.
//
// Activation layout ("padded, channel-blocked"): a level of D x H x W voxels
// is stored with a one-voxel zero halo, Dp x Hp x Wp = (D+2)(H+2)(W+2) rows
// r = z Hp Wp + y Wp + x in padded coordinates, followed by kSlack zero rows;
// channels are in blocks of 8: tensor[g][r][8] (bf16), one 16-byte row per
// (block, voxel). A 3x3x3 tap (a, b, c) of voxel row r reads input row
// r + (a-1) Hp Wp + (b-1) Wp + (c-1): every tap is a shift of whole rows, so the
// convolution is an implicit GEMM whose A operand for one tap is a contiguous
// range of 16-byte rows (a K-major no-swizzle tensor-core operand whose start
// moves by 16 bytes per row). Halo and slack rows hold zeros (the zero padding
// of the convolution); kernels write interior rows only.
#pragma once
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace unet {

constexpr int kSlack = 1024;      // zero rows after the padded volume (>= 128 x tiles per CTA, >= K chunk)
constexpr int kMaxTiles = 8;      // 128-row tiles per convolution CTA
constexpr int kMaxStages = 6;     // pipeline buffers
constexpr int kConvThreads = 128;

struct Vol {
  int D, H, W;       // interior voxels
  int Dp, Hp, Wp;    // padded
  long long P;       // Hp * Wp
  long long npad;    // Dp * P
  long long rows;    // rows per channel block (npad + kSlack)
  long long r_begin; // first interior row (1, 1, 1)
  long long r_end;   // last interior row + 1
};

inline Vol make_vol(int D, int H, int W) {
  Vol v;
  v.D = D; v.H = H; v.W = W;
  v.Dp = D + 2; v.Hp = H + 2; v.Wp = W + 2;
  v.P = (long long)v.Hp * v.Wp;
  v.npad = (long long)v.Dp * v.P;
  v.rows = v.npad + kSlack;
  v.r_begin = v.P + v.Wp + 1;
  v.r_end = (long long)D * v.P + (long long)H * v.Wp + W + 1;
  return v;
}

// 3x3x3 convolution (forward, or data gradient with the flipped transposed
// weight image): out[r][co] = sum_{tap, ci} in[r + off(tap)][ci] w[tap][co][ci]
struct ConvArgs {
  const __nv_bfloat16* src0;
  const __nv_bfloat16* src1;
  int nchunk;   // input chunks of 16 channels
  int nchunk0;  // chunks taken from src0 (blocks 2c, 2c+1); the rest from src1
  const __nv_bfloat16* wimg;  // [3][nchunk][9][2][cout][8]
  int cout;
  __nv_bfloat16* dst0;
  __nv_bfloat16* dst1;
  int dgroups0;  // output blocks [0, dgroups0) to dst0, the rest to dst1
  const __nv_bfloat16* mask0;  // optional: output zeroed where this tensor is <= 0 (same split)
  const __nv_bfloat16* mask1;
  int relu;
  Vol v;
  int T;        // 128-row tiles per CTA
  int nstage;   // pipeline buffers
  int R;        // rows of an input slab: 128 T + 2 Wp + 2
  uint32_t a_bytes, b_bytes, stage_bytes;
  uint32_t tmem_cols;
  int* err;
};

// The same convolution with the input planes streamed through a CTA that owns
// T in-plane tiles of Zc output planes (cout <= 64): for input plane p, in-plane
// tap (dy, dx) and a 16-channel chunk one MMA with N = (number of valid dz) x
// cout adds in[p] w[dz][dy][dx] to output planes p + 1 - dz at once (adjacent
// TMEM column blocks), so each input tile is read once for up to three taps.
struct ConvZArgs {
  ConvArgs c;             // sources, outputs, masks, geometry, T, R, stage sizes (a_bytes), tmem_cols, err
  const __nv_bfloat16* zimg;  // [nchunk][9 (dy, dx)][2][3 cout (dz, co)][8]
  int Zc;                 // output planes per CTA
  long long u_begin, u_end;  // in-plane rows of the interior: Wp + 1 .. H Wp + W + 1
  uint32_t bz_bytes;      // one chunk's image: 9 x 2 x 3 cout x 16
  uint32_t a_region;      // nstage x a_bytes (B buffers follow)
};

// weight gradient of a 3x3x3 convolution:
// dw[tap][co][ci] += sum_r in[r + off(tap)][ci] dz[r][co]
struct WgradArgs {
  const __nv_bfloat16* src0;
  const __nv_bfloat16* src1;
  int gin, gin0;  // input channel blocks; [0, gin0) from src0
  const __nv_bfloat16* dz;
  int cout, cin;  // cin = 8 gin
  float* dw;      // [27][cout][cin]
  Vol v;
  int Kc;         // rows per chunk (multiple of 16)
  long long nchunks;
  int taps;       // taps per CTA: 9 (one dz) or 3 (one dz, dy)
  int R;          // Kc + 2 Wp + 2
  int nstage;
  uint32_t x_bytes, dz_bytes;  // per stage
  uint32_t x_region, smem_main;
  uint32_t tmem_cols;
  int* err;
};

// error bits written by the kernels
enum { kErrWaitProducer = 1, kErrWaitMma = 2, kErrWaitDone = 4 };

void launch_conv3(const ConvArgs& a, cudaStream_t s);
void launch_conv3z(const ConvZArgs& a, cudaStream_t s);
void launch_wgrad(const WgradArgs& a, cudaStream_t s);
uint64_t launch_count();

}  // namespace unet
