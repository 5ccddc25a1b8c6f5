// unet_api.cu -- host side of the U-Net warm start: the network's buffers,
// forward and backward passes, masked MSE loss, Adam, training samples, the
// warm start of the Poisson solve, and the unet_* C ABI (include/unet.h).
//
// Layer table (written for the library; the oracle keeps its own): two 3x3x3
// convolutions with ReLU per level, channels 16/32/64/128, 2x2x2 average
// pooling down, nearest x2 upsampling and concatenation [upsampled, skip] up,
// a 1x1x1 output convolution, no biases. The input's 2 channels are stored as
// one 16-channel chunk (channels 2..15 zero, their weights zero).
// Elementwise kernels (input packing, pooling, upsampling, their adjoints, the
// output layer and the loss) run on CUDA cores: they move a few bytes per voxel.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/unet.h"
#include "dev_mem.cuh"
#include "unet_internal.cuh"
#include "unet_warm.cuh"

namespace unet {

struct LayerDef {
  const char* name;
  int cin, cout, level;
};
// forward order
static const LayerDef kLayers[] = {
    {"e0a", 2, 16, 0},   {"e0b", 16, 16, 0},  {"e1a", 16, 32, 1},  {"e1b", 32, 32, 1},  {"e2a", 32, 64, 2},
    {"e2b", 64, 64, 2},  {"e3a", 64, 128, 3}, {"e3b", 128, 128, 3}, {"d2a", 192, 64, 2}, {"d2b", 64, 64, 2},
    {"d1a", 96, 32, 1},  {"d1b", 32, 32, 1},  {"d0a", 48, 16, 0},  {"d0b", 16, 16, 0},
};
constexpr int kNL = 14;
constexpr int kOutC = 16;
enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, D0A, D0B };

int64_t num_weights() {
  int64_t n = 0;
  for (auto& l : kLayers) n += 27ll * l.cin * l.cout;
  return n + kOutC;
}

struct Tensor {
  __nv_bfloat16* p = nullptr;
  int C = 0, level = 0;
};

struct Layer {
  LayerDef def;
  int cin;  // stored input channels (multiple of 16)
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // [27][cout][cin]
  __nv_bfloat16* wf = nullptr;  // forward image [3][cin/16][9][2][cout][8]
  __nv_bfloat16* wd = nullptr;  // data-gradient image [3][cout/16][9][2][cin][8]
  __nv_bfloat16* zf = nullptr;  // the forward image with dz next to the output channel: [cin/16][9][2][3][cout][8]
  __nv_bfloat16* zd = nullptr;  // the same for the data-gradient image: [cout/16][9][2][3][cin][8]
  long long nw() const { return 27ll * def.cout * cin; }
};

}  // namespace unet

struct unet_handle {
  int D = 0, H = 0, W = 0;
  unet::Vol vol[4];
  cudaStream_t stream = nullptr;
  unet::Layer L[unet::kNL];
  float *wout = nullptr, *gout = nullptr, *mout = nullptr, *vout = nullptr;
  float* wbuf = nullptr;  // all master weights, then gradients, m, v (each n_store floats)
  long long n_store = 0;
  // activations (padded blocked layout)
  unet::Tensor X, E0A, E0, U0, D0A, D0, P1, E1A, E1, U1, D1A, D1, P2, E2A, E2, U2, D2A, D2, P3, E3A, E3;
  // gradients
  unet::Tensor GD0, GD0A, GU0, GE0S, GE0, GE0A, GD1, GD1A, GU1, GE1S, GP1, GE1, GE1A, GD2, GD2A, GU2, GE2S, GP2, GE2,
      GE2A, GE3, GE3A, GP3;
  std::vector<void*> allocs;
  float* y = nullptr;       // D x H x W output of the last forward
  float* dy = nullptr;      // scratch output gradient
  float* xin = nullptr;     // 2 x D x H x W input scratch (warm start)
  double* red = nullptr;    // device reductions: [0] loss, [1] sum of squares, [2] scale s
  int* err = nullptr;
  long long adam_t = 0;
  bool have_forward = false;
  // per-layer forward timing (unet_set_profiling): events around each convolution
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double layer_ms[14] = {0};
  long long layer_n[14] = {0};
  char msg[256] = {0};
};

namespace unet {

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long vrow(const Vol& v, int d, int j, int i) {
  return (long long)(d + 1) * v.P + (long long)(j + 1) * v.Wp + (i + 1);
}

__device__ __forceinline__ void unpack8(uint4 u, float* f) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    f[2 * j] = __uint_as_float(w[j] << 16);
    f[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
  }
}
__device__ __forceinline__ uint32_t pk2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint4 pack8(const float* f) {
  return make_uint4(pk2(f[0], f[1]), pk2(f[2], f[3]), pk2(f[4], f[5]), pk2(f[6], f[7]));
}
__device__ __forceinline__ uint4 ld_row(const __nv_bfloat16* t, const Vol& v, int g, long long r) {
  return *reinterpret_cast<const uint4*>(t + ((long long)g * v.rows + r) * 8);
}
__device__ __forceinline__ void st_row(__nv_bfloat16* t, const Vol& v, int g, long long r, uint4 u) {
  *reinterpret_cast<uint4*>(t + ((long long)g * v.rows + r) * 8) = u;
}

#define VOXELS(v, n)                                                                              \
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < (long long)(v).D * (v).H * (v).W; \
       n += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ void decode(const Vol& v, long long n, int& d, int& j, int& i) {
  const long long hw = (long long)v.H * v.W;
  d = (int)(n / hw);
  const long long rem = n - (long long)d * hw;
  j = (int)(rem / v.W);
  i = (int)(rem - (long long)j * v.W);
}

// input (2 channels, dense FP32) -> block 0 of the level-0 input tensor
__global__ void k_pack_x(Vol v, const float* __restrict__ x, __nv_bfloat16* X) {
  const long long nv = (long long)v.D * v.H * v.W;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    float f[8] = {x[n], x[nv + n], 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    st_row(X, v, 0, vrow(v, d, j, i), pack8(f));
  }
}

// out[coarse] = mean of the 8 children (all blocks)
__global__ void k_pool(Vol vf, Vol vc, int G, const __nv_bfloat16* in, __nv_bfloat16* out) {
  VOXELS(vc, n) {
    int d, j, i;
    decode(vc, n, d, j, i);
    for (int g = 0; g < G; ++g) {
      float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int c = 0; c < 8; ++c) {
        float f[8];
        unpack8(ld_row(in, vf, g, vrow(vf, 2 * d + (c >> 2), 2 * j + ((c >> 1) & 1), 2 * i + (c & 1))), f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += f[k];
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] *= 0.125f;
      st_row(out, vc, g, vrow(vc, d, j, i), pack8(acc));
    }
  }
}

// out[fine] = in[parent]
__global__ void k_upsample(Vol vc, Vol vf, int G, const __nv_bfloat16* in, __nv_bfloat16* out) {
  VOXELS(vf, n) {
    int d, j, i;
    decode(vf, n, d, j, i);
    const long long rc = vrow(vc, d >> 1, j >> 1, i >> 1), rf = vrow(vf, d, j, i);
    for (int g = 0; g < G; ++g) st_row(out, vf, g, rf, ld_row(in, vc, g, rc));
  }
}

// adjoint of upsampling: out[coarse] = sum of the 8 children of in
__global__ void k_upsample_back(Vol vf, Vol vc, int G, const __nv_bfloat16* in, __nv_bfloat16* out) {
  VOXELS(vc, n) {
    int d, j, i;
    decode(vc, n, d, j, i);
    for (int g = 0; g < G; ++g) {
      float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int c = 0; c < 8; ++c) {
        float f[8];
        unpack8(ld_row(in, vf, g, vrow(vf, 2 * d + (c >> 2), 2 * j + ((c >> 1) & 1), 2 * i + (c & 1))), f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += f[k];
      }
      st_row(out, vc, g, vrow(vc, d, j, i), pack8(acc));
    }
  }
}

// gradient at an encoder output: out[fine] = (skip[fine] + dp[parent] / 8) where e[fine] > 0
__global__ void k_pool_back(Vol vf, Vol vc, int G, const __nv_bfloat16* skip, const __nv_bfloat16* dp,
                            const __nv_bfloat16* e, __nv_bfloat16* out) {
  VOXELS(vf, n) {
    int d, j, i;
    decode(vf, n, d, j, i);
    const long long rf = vrow(vf, d, j, i), rc = vrow(vc, d >> 1, j >> 1, i >> 1);
    for (int g = 0; g < G; ++g) {
      float s[8], p[8], m[8];
      unpack8(ld_row(skip, vf, g, rf), s);
      unpack8(ld_row(dp, vc, g, rc), p);
      unpack8(ld_row(e, vf, g, rf), m);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] = m[k] > 0.f ? s[k] + 0.125f * p[k] : 0.f;
      st_row(out, vf, g, rf, pack8(s));
    }
  }
}

// output layer: y = sum_c w[c] d0[c]
__global__ void k_out_fwd(Vol v, const __nv_bfloat16* d0, const float* __restrict__ w, float* y) {
  __shared__ float ws[kOutC];
  if (threadIdx.x < kOutC) ws[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    const long long r = vrow(v, d, j, i);
    float a[8], b[8];
    unpack8(ld_row(d0, v, 0, r), a);
    unpack8(ld_row(d0, v, 1, r), b);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += ws[k] * a[k] + ws[8 + k] * b[k];
    y[n] = s;
  }
}

// output layer backward, with dy given (t == nullptr) or from the masked MSE
// loss against t (planes d < loss_planes, n voxels there):
//   dy = 2 (y - t) / n, loss += (y - t)^2 / n;
//   gd0[c] = w[c] dy where d0[c] > 0 ; gw[c] += sum dy d0[c]
__global__ void k_out_back(Vol v, const __nv_bfloat16* d0, const float* __restrict__ w, const float* y,
                           const float* t, int loss_planes, double inv_n, const float* dy_in, __nv_bfloat16* gd0,
                           float* gw, double* loss) {
  __shared__ float ws[kOutC];
  __shared__ float red[kOutC + 1][8];
  if (threadIdx.x < kOutC) ws[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  float acc[kOutC + 1];
#pragma unroll
  for (int k = 0; k <= kOutC; ++k) acc[k] = 0.f;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    float dyv;
    if (t) {
      if (d < loss_planes) {
        const float e = y[n] - t[n];
        dyv = (float)(2.0 * inv_n) * e;
        acc[kOutC] += e * e;
      } else {
        dyv = 0.f;
      }
    } else {
      dyv = dy_in[n];
    }
    const long long r = vrow(v, d, j, i);
    float a[16];
    unpack8(ld_row(d0, v, 0, r), a);
    unpack8(ld_row(d0, v, 1, r), a + 8);
    float o[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      acc[k] += dyv * a[k];
      o[k] = a[k] > 0.f ? ws[k] * dyv : 0.f;
    }
    st_row(gd0, v, 0, r, pack8(o));
    st_row(gd0, v, 1, r, pack8(o + 8));
  }
  // block reduction: warp shuffles, then one lane per warp
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k <= kOutC; ++k) {
    float s = acc[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x <= kOutC) {
    float s = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    if (threadIdx.x < kOutC) atomicAdd(&gw[threadIdx.x], s);
    else if (t) atomicAdd(loss, (double)s * inv_n);
  }
}

// forward weight image: [3 dz][cin/16][9][2][cout][8], element W[tap][co][ci]
__global__ void k_wimage_fwd(const float* __restrict__ w, int cin, int cout, __nv_bfloat16* img) {
  const long long total = 27ll * cin * cout;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total; n += (long long)gridDim.x * blockDim.x) {
    long long q = n;
    const int e = (int)(q % 8); q /= 8;
    const int co = (int)(q % cout); q /= cout;
    const int kg = (int)(q % 2); q /= 2;
    const int t9 = (int)(q % 9); q /= 9;
    const int ch = (int)(q % (cin / 16)); q /= (cin / 16);
    const int dz = (int)q;
    const int ci = ch * 16 + kg * 8 + e;
    img[n] = __float2bfloat16_rn(w[((long long)(dz * 9 + t9) * cout + co) * cin + ci]);
  }
}

// data-gradient image: a convolution from cout to cin channels with the taps
// flipped: [3][cout/16][9][2][cin][8], element W[26 - tap'][co][ci]
__global__ void k_wimage_dgrad(const float* __restrict__ w, int cin, int cout, __nv_bfloat16* img) {
  const long long total = 27ll * cin * cout;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total; n += (long long)gridDim.x * blockDim.x) {
    long long q = n;
    const int e = (int)(q % 8); q /= 8;
    const int ci = (int)(q % cin); q /= cin;
    const int kg = (int)(q % 2); q /= 2;
    const int t9 = (int)(q % 9); q /= 9;
    const int ch = (int)(q % (cout / 16)); q /= (cout / 16);
    const int dz = (int)q;
    const int co = ch * 16 + kg * 8 + e;
    const int tap = 26 - (dz * 9 + t9);
    img[n] = __float2bfloat16_rn(w[((long long)tap * cout + co) * cin + ci]);
  }
}

// image for the plane-streaming convolution: dz moved next to the output channel,
// zimg[c][t9][kg][dz][n][e] = img[dz][c][t9][kg][n][e] (N output channels, nch chunks)
__global__ void k_zimage(const __nv_bfloat16* __restrict__ img, int nch, int N, __nv_bfloat16* zimg) {
  const long long total = 27ll * 16 * nch * N;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    const int e = (int)(r % 8); r /= 8;
    const int n = (int)(r % N); r /= N;
    const int dz = (int)(r % 3); r /= 3;
    const int kg = (int)(r % 2); r /= 2;
    const int t9 = (int)(r % 9); r /= 9;
    const int c = (int)r;
    zimg[q] = img[((((long long)(dz * nch + c) * 9 + t9) * 2 + kg) * N + n) * 8 + e];
  }
}

// Adam (Kingma and Ba, Algorithm 1) over the flat FP32 master weights
__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
}

// training sample, pass 1: delta = phi_new - phi_old on the unknown nodes,
// x0 = A delta (zero Dirichlet planes), t = delta; sum (A delta)^2
__global__ void k_sample_delta(Vol v, const double* __restrict__ pn, const double* __restrict__ po, float* x0, float* t,
                               double* ss) {
  const int nx = v.W, ny = v.H, nz = v.D;  // nodes: (nz + 1) planes
  const long long pl = (long long)nx * ny;
  double acc = 0.0;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    if (d >= nz - 1) {
      x0[n] = 0.f;
      t[n] = 0.f;
      continue;
    }
    const int k = d + 1;
    auto del = [&](int kk, int jj, int ii) -> double {
      if (kk <= 0 || kk >= nz) return 0.0;
      const long long q = (long long)kk * pl + (long long)jj * nx + ii;
      return pn[q] - po[q];
    };
    const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
    const double c = del(k, j, i);
    const double a = 6.0 * c - del(k, j, im) - del(k, j, ip) - del(k, jm, i) - del(k, jp, i) - del(k - 1, j, i) -
                     del(k + 1, j, i);
    x0[n] = (float)a;
    t[n] = (float)c;
    acc += a * a;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(ss, acc);
}

// pass 2: s = sqrt(sum / unknowns); x0 /= s, t /= s, x1 = ramp (d + 1) / nz
__global__ void k_sample_scale(Vol v, const double* ss, double nunk, float* x0, float* x1, float* t, double* s_out) {
  const double s = sqrt(ss[0] / nunk);
  const float inv = s > 0.0 ? (float)(1.0 / s) : 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) s_out[0] = s;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    x0[n] *= inv;
    if (t) t[n] *= inv;
    x1[n] = (float)(d + 1) / (float)v.D;
  }
}

// dense FP32 (C, D, H, W) -> blocked BF16 tensor of G blocks (channels >= C zero)
__global__ void k_pack_dense(Vol v, int C, int G, const float* __restrict__ x, __nv_bfloat16* t) {
  const long long nv = (long long)v.D * v.H * v.W;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    const long long r = vrow(v, d, j, i);
    for (int g = 0; g < G; ++g) {
      float f[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = g * 8 + k < C ? x[(long long)(g * 8 + k) * nv + n] : 0.f;
      st_row(t, v, g, r, pack8(f));
    }
  }
}

// blocked BF16 tensor -> dense FP32 (C, D, H, W)
__global__ void k_unpack_dense(Vol v, int C, const __nv_bfloat16* t, float* x) {
  const long long nv = (long long)v.D * v.H * v.W;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    const long long r = vrow(v, d, j, i);
    for (int g = 0; g * 8 < C; ++g) {
      float f[8];
      unpack8(ld_row(t, v, g, r), f);
      for (int k = 0; k < 8 && g * 8 + k < C; ++k) x[(long long)(g * 8 + k) * nv + n] = f[k];
    }
  }
}

// residual loss, pass 1: e = x0 - A y on the unknown planes (the last plane is
// the anode: y there counts as 0, e = 0); sum e^2
__device__ __forceinline__ float stencil_A(const Vol& v, const float* __restrict__ f, long long n, int d, int j, int i) {
  const long long hw = (long long)v.H * v.W;
  const int im = i == 0 ? v.W - 1 : i - 1, ip = i == v.W - 1 ? 0 : i + 1;
  const int jm = j == 0 ? v.H - 1 : j - 1, jp = j == v.H - 1 ? 0 : j + 1;
  const long long row = n - i;
  float a = 6.f * f[n] - f[row + im] - f[row + ip] - f[n + (long long)(jm - j) * v.W] - f[n + (long long)(jp - j) * v.W];
  if (d > 0) a -= f[n - hw];
  if (d < v.D - 2) a -= f[n + hw];
  return a;
}

__global__ void k_resid_e(Vol v, const float* __restrict__ x0, const float* __restrict__ y, float* e, double* loss) {
  double acc = 0.0;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    if (d >= v.D - 1) {
      e[n] = 0.f;
      continue;
    }
    const float r = x0[n] - stencil_A(v, y, n, d, j, i);
    e[n] = r;
    acc += (double)r * r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// pass 2: dy = -(2 / n) A e (0 on the anode plane); loss /= n once
__global__ void k_resid_dy(Vol v, const float* __restrict__ e, double inv_n, float* dy, double* loss) {
  if (blockIdx.x == 0 && threadIdx.x == 0) loss[0] *= inv_n;
  const float c = (float)(-2.0 * inv_n);
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    dy[n] = d >= v.D - 1 ? 0.f : c * stencil_A(v, e, n, d, j, i);
  }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
static int grid_for(long long n, int block = 256) {
  long long g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}
#define ULAUNCH(grid, block, smem, stream, ...) (++g_ew_launches), __VA_ARGS__<<<grid, block, smem, stream>>>
static unsigned long long g_ew_launches = 0;

static int pow2_cols(int c) {
  int p = 32;
  while (p < c) p <<= 1;
  return p;
}

// convolution (forward, or data gradient when `dgrad`) of layer l
static cudaEvent_t take_event(unet_handle* n) {
  if (!n->ev_pool.empty()) {
    cudaEvent_t e = n->ev_pool.back();
    n->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// sums the timed forward convolutions whose events have completed
static void collect_times(unet_handle* n) {
  for (auto& p : n->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
      n->layer_ms[p.first] += ms;
      n->layer_n[p.first] += 1;
    }
    n->ev_pool.push_back(p.second.first);
    n->ev_pool.push_back(p.second.second);
  }
  n->ev_pending.clear();
}

static void conv_impl(unet_handle* n, int l, bool dgrad, const Tensor& s0, const Tensor* s1, const Tensor& d0,
                      const Tensor* d1, const Tensor* m0, const Tensor* m1, bool relu, cudaStream_t st);

static void conv(unet_handle* n, int l, bool dgrad, const Tensor& s0, const Tensor* s1, const Tensor& d0,
                 const Tensor* d1, const Tensor* m0, const Tensor* m1, bool relu, cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (n->prof && !dgrad) cudaStreamIsCapturing(st, &cap);
  if (!n->prof || dgrad || cap != cudaStreamCaptureStatusNone) {  // never timed inside a recorded graph
    conv_impl(n, l, dgrad, s0, s1, d0, d1, m0, m1, relu, st);
    return;
  }
  cudaEvent_t a = take_event(n), b = take_event(n);
  cudaEventRecord(a, st);
  conv_impl(n, l, dgrad, s0, s1, d0, d1, m0, m1, relu, st);
  cudaEventRecord(b, st);
  n->ev_pending.push_back({l, {a, b}});
}

// Plane streaming for 16 output channels (the finest level): there it reads each
// input tile once for three dz taps; at 32 and 64 channels (coarser levels, one
// 128-row tile per CTA) the per-plane kernel measured faster.
constexpr int kZMaxCout = 16;

static void conv_impl(unet_handle* n, int l, bool dgrad, const Tensor& s0, const Tensor* s1, const Tensor& d0,
                      const Tensor* d1, const Tensor* m0, const Tensor* m1, bool relu, cudaStream_t st) {
  const Layer& L = n->L[l];
  if ((dgrad ? L.cin : L.def.cout) <= kZMaxCout) {
    const int cin = dgrad ? L.def.cout : L.cin;
    const int cout = dgrad ? L.cin : L.def.cout;
    const Vol& v = n->vol[s0.level];
    ConvZArgs z{};
    ConvArgs& a = z.c;
    a.src0 = s0.p;
    a.src1 = s1 ? s1->p : nullptr;
    a.nchunk = cin / 16;
    a.nchunk0 = s1 ? s0.C / 16 : a.nchunk;
    a.cout = cout;
    a.dst0 = d0.p;
    a.dst1 = d1 ? d1->p : nullptr;
    a.dgroups0 = d1 ? d0.C / 8 : cout / 8;
    a.mask0 = m0 ? m0->p : nullptr;
    a.mask1 = m1 ? m1->p : nullptr;
    a.relu = relu ? 1 : 0;
    a.v = v;
    a.err = n->err;
    z.zimg = dgrad ? L.zd : L.zf;
    // TMEM T x Zc x cout <= 256 columns (two CTAs per SM): the deepest plane column
    // that leaves at least one tile, then two tiles where that still keeps 8 planes
    a.T = cout <= 16 ? 2 : 1;
    z.Zc = 256 / (a.T * cout);
    if (z.Zc > 8) z.Zc = 8;
    if (z.Zc > v.D) z.Zc = v.D;
    a.R = 128 * a.T + 2 * v.Wp + 2;
    a.a_bytes = (uint32_t)a.R * 32u;
    z.bz_bytes = 9u * 2u * 3u * (uint32_t)cout * 16u;
    int ns = (int)((110u * 1024u - 2u * z.bz_bytes) / a.a_bytes);
    a.nstage = ns > 4 ? 4 : (ns < 2 ? 2 : ns);
    z.a_region = (uint32_t)a.nstage * a.a_bytes;
    a.stage_bytes = a.a_bytes;
    a.tmem_cols = (uint32_t)pow2_cols(a.T * z.Zc * cout);
    z.u_begin = v.Wp + 1;
    z.u_end = (long long)v.H * v.Wp + v.W + 1;
    launch_conv3z(z, st);
    return;
  }
  ConvArgs a{};
  const int cin = dgrad ? L.def.cout : L.cin;
  const int cout = dgrad ? L.cin : L.def.cout;
  const Vol& v = n->vol[s0.level];
  a.src0 = s0.p;
  a.src1 = s1 ? s1->p : nullptr;
  a.nchunk = cin / 16;
  a.nchunk0 = s1 ? s0.C / 16 : a.nchunk;
  a.wimg = dgrad ? L.wd : L.wf;
  a.cout = cout;
  a.dst0 = d0.p;
  a.dst1 = d1 ? d1->p : nullptr;
  a.dgroups0 = d1 ? d0.C / 8 : cout / 8;
  a.mask0 = m0 ? m0->p : nullptr;
  a.mask1 = m1 ? m1->p : nullptr;
  a.relu = relu ? 1 : 0;
  a.v = v;
  // tiles per CTA: TMEM columns T * cout <= 256, at most kMaxTiles; stages of
  // (2 x R input rows + weight image) within about 100 KB so that two CTAs
  // share an SM (one overlaps its epilogue with the other's MMAs)
  int T = 256 / cout;
  if (T < 1) T = 1;
  if (T > kMaxTiles) T = kMaxTiles;
  int ns = 0;
  uint32_t stage = 0;
  for (;; T /= 2) {
    a.R = 128 * T + 2 * v.Wp + 2;
    a.a_bytes = (uint32_t)a.R * 32u;
    a.b_bytes = (uint32_t)(9 * 2 * cout * 16);
    stage = ((a.a_bytes + a.b_bytes + 127u) / 128u) * 128u;
    ns = (int)(100u * 1024u / stage);
    if (ns >= 2 || T == 1) break;
  }
  ns = ns > 4 ? 4 : (ns < 2 ? 2 : ns);
  a.T = T;
  a.nstage = ns;
  a.stage_bytes = stage;
  a.tmem_cols = (uint32_t)pow2_cols(T * cout);
  a.err = n->err;
  launch_conv3(a, st);
}

static void wgrad(unet_handle* n, int l, const Tensor& s0, const Tensor* s1, const Tensor& dz, cudaStream_t st) {
  Layer& L = n->L[l];
  WgradArgs a{};
  const Vol& v = n->vol[s0.level];
  a.src0 = s0.p;
  a.src1 = s1 ? s1->p : nullptr;
  a.gin = L.cin / 8;
  a.gin0 = s1 ? s0.C / 8 : a.gin;
  a.dz = dz.p;
  a.cout = L.def.cout;
  a.cin = L.cin;
  a.dw = L.g;
  a.v = v;
  a.taps = 9 * a.cout <= 288 ? 9 : 3;
  a.tmem_cols = (uint32_t)pow2_cols(a.taps * a.cout);
  const int ngmax = a.gin < 16 ? a.gin : 16;
  for (a.Kc = 256;; a.Kc /= 2) {
    a.R = a.Kc + 2 * v.Wp + 2;
    a.nstage = 2;
    a.x_bytes = (uint32_t)ngmax * a.R * 16u;
    a.dz_bytes = (uint32_t)(a.cout / 8) * a.Kc * 16u;
    const uint32_t xr1 = (uint32_t)a.nstage * a.x_bytes;
    const uint32_t xr2 = (uint32_t)(a.nstage - 1) * a.x_bytes + 16u * a.R * 16u;
    a.x_region = ((xr1 > xr2 ? xr1 : xr2) + 127u) / 128u * 128u;
    a.smem_main = a.x_region + (uint32_t)a.nstage * a.dz_bytes;
    if (a.smem_main <= 200u * 1024u || a.Kc == 16) break;
  }
  a.nchunks = (v.r_end - v.r_begin + a.Kc - 1) / a.Kc;
  a.err = n->err;
  launch_wgrad(a, st);
}

static void rebuild_images(unet_handle* n, cudaStream_t st) {
  for (int l = 0; l < kNL; ++l) {
    Layer& L = n->L[l];
    const long long tot = L.nw();
    ULAUNCH(grid_for(tot), 256, 0, st, k_wimage_fwd)(L.w, L.cin, L.def.cout, L.wf);
    ULAUNCH(grid_for(tot), 256, 0, st, k_wimage_dgrad)(L.w, L.cin, L.def.cout, L.wd);
    if (L.def.cout <= kZMaxCout) ULAUNCH(grid_for(tot), 256, 0, st, k_zimage)(L.wf, L.cin / 16, L.def.cout, L.zf);
    if (L.cin <= kZMaxCout) ULAUNCH(grid_for(tot), 256, 0, st, k_zimage)(L.wd, L.def.cout / 16, L.cin, L.zd);
  }
}

static cudaError_t forward(unet_handle* n, const float* x, float* y, cudaStream_t st) {
  const Vol* V = n->vol;
  ULAUNCH(grid_for((long long)V[0].D * V[0].H * V[0].W), 256, 0, st, k_pack_x)(V[0], x, n->X.p);
  conv(n, E0A, false, n->X, nullptr, n->E0A, nullptr, nullptr, nullptr, true, st);
  conv(n, E0B, false, n->E0A, nullptr, n->E0, nullptr, nullptr, nullptr, true, st);
  ULAUNCH(grid_for((long long)V[1].D * V[1].H * V[1].W), 256, 0, st, k_pool)(V[0], V[1], 2, n->E0.p, n->P1.p);
  conv(n, E1A, false, n->P1, nullptr, n->E1A, nullptr, nullptr, nullptr, true, st);
  conv(n, E1B, false, n->E1A, nullptr, n->E1, nullptr, nullptr, nullptr, true, st);
  ULAUNCH(grid_for((long long)V[2].D * V[2].H * V[2].W), 256, 0, st, k_pool)(V[1], V[2], 4, n->E1.p, n->P2.p);
  conv(n, E2A, false, n->P2, nullptr, n->E2A, nullptr, nullptr, nullptr, true, st);
  conv(n, E2B, false, n->E2A, nullptr, n->E2, nullptr, nullptr, nullptr, true, st);
  ULAUNCH(grid_for((long long)V[3].D * V[3].H * V[3].W), 256, 0, st, k_pool)(V[2], V[3], 8, n->E2.p, n->P3.p);
  conv(n, E3A, false, n->P3, nullptr, n->E3A, nullptr, nullptr, nullptr, true, st);
  conv(n, E3B, false, n->E3A, nullptr, n->E3, nullptr, nullptr, nullptr, true, st);
  ULAUNCH(grid_for((long long)V[2].D * V[2].H * V[2].W), 256, 0, st, k_upsample)(V[3], V[2], 16, n->E3.p, n->U2.p);
  conv(n, D2A, false, n->U2, &n->E2, n->D2A, nullptr, nullptr, nullptr, true, st);
  conv(n, D2B, false, n->D2A, nullptr, n->D2, nullptr, nullptr, nullptr, true, st);
  ULAUNCH(grid_for((long long)V[1].D * V[1].H * V[1].W), 256, 0, st, k_upsample)(V[2], V[1], 8, n->D2.p, n->U1.p);
  conv(n, D1A, false, n->U1, &n->E1, n->D1A, nullptr, nullptr, nullptr, true, st);
  conv(n, D1B, false, n->D1A, nullptr, n->D1, nullptr, nullptr, nullptr, true, st);
  ULAUNCH(grid_for((long long)V[0].D * V[0].H * V[0].W), 256, 0, st, k_upsample)(V[1], V[0], 4, n->D1.p, n->U0.p);
  conv(n, D0A, false, n->U0, &n->E0, n->D0A, nullptr, nullptr, nullptr, true, st);
  conv(n, D0B, false, n->D0A, nullptr, n->D0, nullptr, nullptr, nullptr, true, st);
  ULAUNCH(grid_for((long long)V[0].D * V[0].H * V[0].W), 256, 0, st, k_out_fwd)(V[0], n->D0.p, n->wout, y);
  return cudaGetLastError();
}

// backward from the output gradient (dy given) or from the loss against t
static cudaError_t backward(unet_handle* n, const float* dy, const float* t, int loss_planes, cudaStream_t st) {
  const Vol* V = n->vol;
  cudaError_t e = cudaMemsetAsync(n->wbuf + n->n_store, 0, sizeof(float) * n->n_store, st);  // gradients
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(n->red, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const long long nv0 = (long long)V[0].D * V[0].H * V[0].W;
  const long long nmask = (long long)loss_planes * V[0].H * V[0].W;
  ULAUNCH(grid_for(nv0), 256, 0, st, k_out_back)(V[0], n->D0.p, n->wout, n->y, t, loss_planes,
                                                  nmask > 0 ? 1.0 / (double)nmask : 0.0, dy, n->GD0.p, n->gout, n->red);
  // level 0 decoder
  wgrad(n, D0B, n->D0A, nullptr, n->GD0, st);
  conv(n, D0B, true, n->GD0, nullptr, n->GD0A, nullptr, &n->D0A, nullptr, false, st);
  wgrad(n, D0A, n->U0, &n->E0, n->GD0A, st);
  conv(n, D0A, true, n->GD0A, nullptr, n->GU0, &n->GE0S, &n->U0, &n->E0, false, st);
  ULAUNCH(grid_for((long long)V[1].D * V[1].H * V[1].W), 256, 0, st, k_upsample_back)(V[0], V[1], 4, n->GU0.p, n->GD1.p);
  // level 1 decoder
  wgrad(n, D1B, n->D1A, nullptr, n->GD1, st);
  conv(n, D1B, true, n->GD1, nullptr, n->GD1A, nullptr, &n->D1A, nullptr, false, st);
  wgrad(n, D1A, n->U1, &n->E1, n->GD1A, st);
  conv(n, D1A, true, n->GD1A, nullptr, n->GU1, &n->GE1S, &n->U1, &n->E1, false, st);
  ULAUNCH(grid_for((long long)V[2].D * V[2].H * V[2].W), 256, 0, st, k_upsample_back)(V[1], V[2], 8, n->GU1.p, n->GD2.p);
  // level 2 decoder
  wgrad(n, D2B, n->D2A, nullptr, n->GD2, st);
  conv(n, D2B, true, n->GD2, nullptr, n->GD2A, nullptr, &n->D2A, nullptr, false, st);
  wgrad(n, D2A, n->U2, &n->E2, n->GD2A, st);
  conv(n, D2A, true, n->GD2A, nullptr, n->GU2, &n->GE2S, &n->U2, &n->E2, false, st);
  ULAUNCH(grid_for((long long)V[3].D * V[3].H * V[3].W), 256, 0, st, k_upsample_back)(V[2], V[3], 16, n->GU2.p, n->GE3.p);
  // level 3
  wgrad(n, E3B, n->E3A, nullptr, n->GE3, st);
  conv(n, E3B, true, n->GE3, nullptr, n->GE3A, nullptr, &n->E3A, nullptr, false, st);
  wgrad(n, E3A, n->P3, nullptr, n->GE3A, st);
  conv(n, E3A, true, n->GE3A, nullptr, n->GP3, nullptr, nullptr, nullptr, false, st);
  ULAUNCH(grid_for((long long)V[2].D * V[2].H * V[2].W), 256, 0, st, k_pool_back)(V[2], V[3], 8, n->GE2S.p, n->GP3.p,
                                                                                   n->E2.p, n->GE2.p);
  // level 2 encoder
  wgrad(n, E2B, n->E2A, nullptr, n->GE2, st);
  conv(n, E2B, true, n->GE2, nullptr, n->GE2A, nullptr, &n->E2A, nullptr, false, st);
  wgrad(n, E2A, n->P2, nullptr, n->GE2A, st);
  conv(n, E2A, true, n->GE2A, nullptr, n->GP2, nullptr, nullptr, nullptr, false, st);
  ULAUNCH(grid_for((long long)V[1].D * V[1].H * V[1].W), 256, 0, st, k_pool_back)(V[1], V[2], 4, n->GE1S.p, n->GP2.p,
                                                                                   n->E1.p, n->GE1.p);
  // level 1 encoder
  wgrad(n, E1B, n->E1A, nullptr, n->GE1, st);
  conv(n, E1B, true, n->GE1, nullptr, n->GE1A, nullptr, &n->E1A, nullptr, false, st);
  wgrad(n, E1A, n->P1, nullptr, n->GE1A, st);
  conv(n, E1A, true, n->GE1A, nullptr, n->GP1, nullptr, nullptr, nullptr, false, st);
  ULAUNCH(grid_for(nv0), 256, 0, st, k_pool_back)(V[0], V[1], 2, n->GE0S.p, n->GP1.p, n->E0.p, n->GE0.p);
  // level 0 encoder
  wgrad(n, E0B, n->E0A, nullptr, n->GE0, st);
  conv(n, E0B, true, n->GE0, nullptr, n->GE0A, nullptr, &n->E0A, nullptr, false, st);
  wgrad(n, E0A, n->X, nullptr, n->GE0A, st);
  return cudaGetLastError();
}

static pic_status fail(unet_handle* n, pic_status s, const char* fmt, ...) {
  static char global_msg[256];
  char* dst = n ? n->msg : global_msg;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return s;
}

static pic_status check_err(unet_handle* n) {
  int e = 0;
  if (cudaMemcpyAsync(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet: CUDA error %s", cudaGetErrorString(cudaGetLastError()));
  if (e) return fail(n, PIC_ETIMEOUT, "unet: a tensor-core kernel gave up waiting (error bits %d)", e);
  return PIC_OK;
}

// host flat (oracle order: w[co][ci][a][b][c] per layer, then out) <-> device [27][cout][cin_store]
static void host_to_store(const LayerDef& d, int cin_s, const float* src, std::vector<float>& dst) {
  dst.assign(27ull * d.cout * cin_s, 0.f);
  for (int co = 0; co < d.cout; ++co)
    for (int ci = 0; ci < d.cin; ++ci)
      for (int t = 0; t < 27; ++t) dst[((size_t)t * d.cout + co) * cin_s + ci] = src[((size_t)co * d.cin + ci) * 27 + t];
}
static void store_to_host(const LayerDef& d, int cin_s, const float* src, float* dst) {
  for (int co = 0; co < d.cout; ++co)
    for (int ci = 0; ci < d.cin; ++ci)
      for (int t = 0; t < 27; ++t) dst[((size_t)co * d.cin + ci) * 27 + t] = src[((size_t)t * d.cout + co) * cin_s + ci];
}

static pic_status copy_out(unet_handle* n, const float* dev_base, float* host, int64_t cnt) {
  if (!n || !host || cnt != num_weights()) return fail(n, PIC_EINVAL, "unet: need a handle and %lld values",
                                                        (long long)num_weights());
  std::vector<float> buf(n->n_store);
  if (cudaMemcpyAsync(buf.data(), dev_base, sizeof(float) * n->n_store, cudaMemcpyDeviceToHost, n->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet: copy failed");
  size_t off = 0, hoff = 0;
  for (int l = 0; l < kNL; ++l) {
    const Layer& L = n->L[l];
    store_to_host(L.def, L.cin, buf.data() + off, host + hoff);
    off += L.nw();
    hoff += 27ull * L.def.cin * L.def.cout;
  }
  memcpy(host + hoff, buf.data() + off, sizeof(float) * kOutC);
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// warm start of the PIC solve (FP64 store): x += s f(r / s, ramp)
// ---------------------------------------------------------------------------
// r = b - A x over the unknown nodes; dense FP32 into xin[0]; sum r^2
__global__ void k_warm_resid64(Vol v, const double* __restrict__ x, const double* __restrict__ b, float* r_out,
                               double* ss) {
  const int nx = v.W, ny = v.H, nz = v.D;
  const long long pl = (long long)nx * ny;
  double acc = 0.0;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    if (d >= nz - 1) {
      r_out[n] = 0.f;
      continue;
    }
    const long long u = (long long)d * pl + (long long)j * nx + i;  // unknown index (plane k = d + 1)
    const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
    const long long row = u - i;
    double s = x[row + im] + x[row + ip] + x[u + (long long)(jm - j) * nx] + x[u + (long long)(jp - j) * nx];
    if (d > 0) s += x[u - pl];
    if (d < nz - 2) s += x[u + pl];
    const double r = b[u] - (6.0 * x[u] - s);
    r_out[n] = (float)r;
    acc += r * r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(ss, acc);
}

// x += s y on the unknown nodes
__global__ void k_warm_apply64(Vol v, const double* s_dev, const float* __restrict__ y, double* x) {
  const double s = s_dev[0];
  const long long pl = (long long)v.W * v.H;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    if (d >= v.D - 1) continue;
    x[(long long)d * pl + (long long)j * v.W + i] += s * (double)y[n];
  }
}

// mixed store: phi = vacuum ramp + hi + lo, and A (vacuum ramp) equals the folded
// electrode terms, so r = f - A (hi + lo) with zero values on the electrode
// planes, in FP32 (hi over the unknown view of phi32, lo over the unknowns);
// dense into r_out; sum r^2. (With an external circuit the anode's offset from
// the configured voltage is a further folded term, left out here: it only
// makes this starting residual, not the solve, approximate.)
__global__ void k_warm_resid32(Vol v, const float* __restrict__ hi, const float* __restrict__ lo,
                               const float* __restrict__ f, float* r_out, double* ss) {
  const int nx = v.W, ny = v.H, nz = v.D;
  const long long pl = (long long)nx * ny;
  double acc = 0.0;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    if (d >= nz - 1) {
      r_out[n] = 0.f;
      continue;
    }
    const long long u = (long long)d * pl + (long long)j * nx + i;
    const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
    const long long row = u - i;
    auto X = [&](long long q) { return hi[q] + lo[q]; };
    float s = X(row + im) + X(row + ip) + X(u + (long long)(jm - j) * nx) + X(u + (long long)(jp - j) * nx);
    if (d > 0) s += X(u - pl);
    if (d < nz - 2) s += X(u + pl);
    const float r = f[u] - (6.f * X(u) - s);
    r_out[n] = r;
    acc += (double)r * r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(ss, acc);
}

__global__ void k_warm_apply32(Vol v, const double* s_dev, const float* __restrict__ y, float* hi) {
  const float s = (float)s_dev[0];
  const long long pl = (long long)v.W * v.H;
  VOXELS(v, n) {
    int d, j, i;
    decode(v, n, d, j, i);
    if (d >= v.D - 1) continue;
    hi[(long long)d * pl + (long long)j * v.W + i] += s * y[n];
  }
}

bool warm_matches(const unet_handle* n, int nx, int ny, int nz) { return n->W == nx && n->H == ny && n->D == nz; }

cudaError_t warm_start(unet_handle* n, const WarmTarget& w, cudaStream_t st) {
  const Vol& v = n->vol[0];
  const long long nv = (long long)v.D * v.H * v.W;
  float* r = n->xin;
  float* ramp = n->xin + nv;
  cudaError_t e = cudaMemsetAsync(n->red + 1, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (w.x64)
    ULAUNCH(grid_for(nv), 256, 0, st, k_warm_resid64)(v, w.x64, w.b64, r, n->red + 1);
  else
    ULAUNCH(grid_for(nv), 256, 0, st, k_warm_resid32)(v, w.hi, w.lo, w.f32, r, n->red + 1);
  // scale the residual by its root mean square over the unknowns, ramp in channel 1
  ULAUNCH(grid_for(nv), 256, 0, st, k_sample_scale)(v, n->red + 1, (double)(v.D - 1) * v.H * v.W, r, ramp, nullptr,
                                                    n->red + 2);
  e = forward(n, n->xin, n->y, st);
  if (e != cudaSuccess) return e;
  if (w.x64)
    ULAUNCH(grid_for(nv), 256, 0, st, k_warm_apply64)(v, n->red + 2, n->y, w.x64);
  else
    ULAUNCH(grid_for(nv), 256, 0, st, k_warm_apply32)(v, n->red + 2, n->y, w.hi);
  return cudaGetLastError();
}

}  // namespace unet

using namespace unet;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int64_t unet_num_weights(void) { return num_weights(); }

extern "C" const char* unet_last_error(unet_handle* n) {
  static const char* none = "unet: null handle";
  return n ? n->msg : none;
}

extern "C" uint64_t unet_launch_count(void) { return unet::launch_count() + unet::g_ew_launches; }

extern "C" pic_status unet_create(int32_t D, int32_t H, int32_t W, void* cuda_stream, unet_handle** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (D < 8 || H < 8 || W < 8 || D % 8 || H % 8 || W % 8 || W > 512 || H > 4096 || D > 4096) return PIC_EINVAL;
  unet_handle* n = new unet_handle();
  pic::dev_handle_opened();
  n->D = D;
  n->H = H;
  n->W = W;
  n->stream = (cudaStream_t)cuda_stream;
  for (int l = 0; l < 4; ++l) n->vol[l] = make_vol(D >> l, H >> l, W >> l);
  auto dev_alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (pic::dev_malloc(&p, bytes) != cudaSuccess) return nullptr;
    n->allocs.push_back(p);
    if (cudaMemsetAsync(p, 0, bytes, n->stream) != cudaSuccess) return nullptr;
    return p;
  };
  bool ok = true;
  // weights: every layer's master copy, then gradients, m, v of the same size
  long long ns = 0;
  for (int l = 0; l < kNL; ++l) {
    n->L[l].def = kLayers[l];
    n->L[l].cin = kLayers[l].cin < 16 ? 16 : kLayers[l].cin;
    ns += n->L[l].nw();
  }
  ns += kOutC;
  n->n_store = ns;
  n->wbuf = (float*)dev_alloc(sizeof(float) * 4 * ns);
  ok = ok && n->wbuf;
  if (ok) {
    long long off = 0;
    for (int l = 0; l < kNL; ++l) {
      Layer& L = n->L[l];
      L.w = n->wbuf + off;
      L.g = n->wbuf + ns + off;
      L.m = n->wbuf + 2 * ns + off;
      L.v = n->wbuf + 3 * ns + off;
      off += L.nw();
      L.wf = (__nv_bfloat16*)dev_alloc(sizeof(__nv_bfloat16) * L.nw());
      L.wd = (__nv_bfloat16*)dev_alloc(sizeof(__nv_bfloat16) * L.nw());
      L.zf = (__nv_bfloat16*)dev_alloc(sizeof(__nv_bfloat16) * L.nw());
      L.zd = (__nv_bfloat16*)dev_alloc(sizeof(__nv_bfloat16) * L.nw());
      ok = ok && L.wf && L.wd && L.zf && L.zd;
    }
    n->wout = n->wbuf + off;
    n->gout = n->wbuf + ns + off;
    n->mout = n->wbuf + 2 * ns + off;
    n->vout = n->wbuf + 3 * ns + off;
  }
  auto tensor = [&](Tensor& t, int C, int level) {
    t.C = C;
    t.level = level;
    t.p = (__nv_bfloat16*)dev_alloc(sizeof(__nv_bfloat16) * 8ull * (C / 8) * n->vol[level].rows);
    ok = ok && t.p;
  };
  tensor(n->X, 16, 0);
  tensor(n->E0A, 16, 0); tensor(n->E0, 16, 0); tensor(n->U0, 32, 0); tensor(n->D0A, 16, 0); tensor(n->D0, 16, 0);
  tensor(n->P1, 16, 1); tensor(n->E1A, 32, 1); tensor(n->E1, 32, 1); tensor(n->U1, 64, 1); tensor(n->D1A, 32, 1);
  tensor(n->D1, 32, 1);
  tensor(n->P2, 32, 2); tensor(n->E2A, 64, 2); tensor(n->E2, 64, 2); tensor(n->U2, 128, 2); tensor(n->D2A, 64, 2);
  tensor(n->D2, 64, 2);
  tensor(n->P3, 64, 3); tensor(n->E3A, 128, 3); tensor(n->E3, 128, 3);
  tensor(n->GD0, 16, 0); tensor(n->GD0A, 16, 0); tensor(n->GU0, 32, 0); tensor(n->GE0S, 16, 0); tensor(n->GE0, 16, 0);
  tensor(n->GE0A, 16, 0);
  tensor(n->GD1, 32, 1); tensor(n->GD1A, 32, 1); tensor(n->GU1, 64, 1); tensor(n->GE1S, 32, 1); tensor(n->GP1, 16, 1);
  tensor(n->GE1, 32, 1); tensor(n->GE1A, 32, 1);
  tensor(n->GD2, 64, 2); tensor(n->GD2A, 64, 2); tensor(n->GU2, 128, 2); tensor(n->GE2S, 64, 2); tensor(n->GP2, 32, 2);
  tensor(n->GE2, 64, 2); tensor(n->GE2A, 64, 2);
  tensor(n->GE3, 128, 3); tensor(n->GE3A, 128, 3); tensor(n->GP3, 64, 3);
  const long long nv = (long long)D * H * W;
  n->y = (float*)dev_alloc(sizeof(float) * nv);
  n->dy = (float*)dev_alloc(sizeof(float) * nv);
  n->xin = (float*)dev_alloc(sizeof(float) * 2 * nv);
  n->red = (double*)dev_alloc(sizeof(double) * 8);
  n->err = (int*)dev_alloc(sizeof(int) * 4);
  ok = ok && n->y && n->dy && n->xin && n->red && n->err;
  if (ok) rebuild_images(n, n->stream);
  if (!ok || cudaStreamSynchronize(n->stream) != cudaSuccess) {
    unet_destroy(n);
    return ok ? PIC_ECUDA : PIC_ENOMEM;
  }
  *out = n;
  return PIC_OK;
}

extern "C" pic_status unet_set_profiling(unet_handle* n, int32_t on) {
  if (!n) return PIC_EINVAL;
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) return fail(n, PIC_ECUDA, "unet_set_profiling: sync failed");
  collect_times(n);
  n->prof = on != 0;
  for (int l = 0; l < kNL; ++l) {
    n->layer_ms[l] = 0.0;
    n->layer_n[l] = 0;
  }
  return PIC_OK;
}

extern "C" pic_status unet_get_layer_times(unet_handle* n, double* ms, int64_t* count) {
  if (!n) return PIC_EINVAL;
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) return fail(n, PIC_ECUDA, "unet_get_layer_times: sync failed");
  collect_times(n);
  for (int l = 0; l < kNL; ++l) {
    if (ms) ms[l] = n->layer_ms[l];
    if (count) count[l] = n->layer_n[l];
  }
  return PIC_OK;
}

extern "C" pic_status unet_destroy(unet_handle* n) {
  if (!n) return PIC_OK;
  if (n->stream) cudaStreamSynchronize(n->stream);
  collect_times(n);
  for (cudaEvent_t e : n->ev_pool) cudaEventDestroy(e);
  for (void* p : n->allocs) pic::dev_free(p);
  delete n;
  pic::dev_handle_closed();
  return PIC_OK;
}

extern "C" pic_status unet_set_weights(unet_handle* n, const float* host, int64_t cnt) {
  if (!n || !host || cnt != num_weights()) return fail(n, PIC_EINVAL, "unet_set_weights: need %lld values",
                                                       (long long)num_weights());
  std::vector<float> buf;
  std::vector<float> all(n->n_store, 0.f);
  size_t off = 0, hoff = 0;
  for (int l = 0; l < kNL; ++l) {
    const Layer& L = n->L[l];
    host_to_store(L.def, L.cin, host + hoff, buf);
    memcpy(all.data() + off, buf.data(), sizeof(float) * buf.size());
    off += L.nw();
    hoff += 27ull * L.def.cin * L.def.cout;
  }
  memcpy(all.data() + off, host + hoff, sizeof(float) * kOutC);
  if (cudaMemcpyAsync(n->wbuf, all.data(), sizeof(float) * n->n_store, cudaMemcpyHostToDevice, n->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(n->wbuf + 2 * n->n_store, 0, sizeof(float) * 2 * n->n_store, n->stream) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet_set_weights: copy failed");
  n->adam_t = 0;
  rebuild_images(n, n->stream);
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) return fail(n, PIC_ECUDA, "unet_set_weights: CUDA error");
  return PIC_OK;
}

extern "C" pic_status unet_get_weights(unet_handle* n, float* host, int64_t cnt) {
  return copy_out(n, n ? n->wbuf : nullptr, host, cnt);
}

extern "C" pic_status unet_get_grads(unet_handle* n, float* host, int64_t cnt) {
  return copy_out(n, n ? n->wbuf + n->n_store : nullptr, host, cnt);
}

extern "C" pic_status unet_forward(unet_handle* n, const float* x, float* y) {
  if (!n || !x || !y) return fail(n, PIC_EINVAL, "unet_forward: null argument");
  cudaError_t e = forward(n, x, n->y, n->stream);
  if (e == cudaSuccess && y != n->y)
    e = cudaMemcpyAsync(y, n->y, sizeof(float) * (size_t)n->D * n->H * n->W, cudaMemcpyDeviceToDevice, n->stream);
  if (e != cudaSuccess) return fail(n, PIC_ECUDA, "unet_forward: %s", cudaGetErrorString(e));
  n->have_forward = true;
  return check_err(n);
}

extern "C" pic_status unet_backward(unet_handle* n, const float* dy) {
  if (!n || !dy) return fail(n, PIC_EINVAL, "unet_backward: null argument");
  if (!n->have_forward) return fail(n, PIC_ESTATE, "unet_backward: no forward pass to differentiate");
  cudaError_t e = backward(n, dy, nullptr, n->D, n->stream);
  if (e != cudaSuccess) return fail(n, PIC_ECUDA, "unet_backward: %s", cudaGetErrorString(e));
  return check_err(n);
}

extern "C" pic_status unet_train_step(unet_handle* n, const float* x, const float* t, int32_t loss_planes, float lr,
                                      double* loss) {
  if (!n || !x || !t || loss_planes < 1 || loss_planes > n->D || !(lr >= 0.f))
    return fail(n, PIC_EINVAL, "unet_train_step: bad argument");
  cudaStream_t st = n->stream;
  cudaError_t e = forward(n, x, n->y, st);
  if (e == cudaSuccess) e = backward(n, nullptr, t, loss_planes, st);
  if (e != cudaSuccess) return fail(n, PIC_ECUDA, "unet_train_step: %s", cudaGetErrorString(e));
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
  ULAUNCH(grid_for(n->n_store), 256, 0, st, k_adam)(n->wbuf, n->wbuf + n->n_store, n->wbuf + 2 * n->n_store,
                                                    n->wbuf + 3 * n->n_store, n->n_store, lr, b1, b2, 1e-8f, c1, c2);
  rebuild_images(n, st);
  n->have_forward = false;
  if (loss) {
    if (cudaMemcpyAsync(loss, n->red, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return fail(n, PIC_ECUDA, "unet_train_step: loss read failed");
  }
  return check_err(n);
}

namespace {
struct Scratch {
  std::vector<void*> p;
  ~Scratch() {
    for (void* q : p) pic::dev_free(q);
  }
  Tensor tensor(const Vol& v, int C, int level, cudaStream_t st) {
    Tensor t;
    t.C = C;
    t.level = level;
    const size_t bytes = sizeof(__nv_bfloat16) * 8ull * (C / 8) * v.rows;
    if (pic::dev_malloc((void**)&t.p, bytes) != cudaSuccess) {
      t.p = nullptr;
      return t;
    }
    p.push_back(t.p);
    cudaMemsetAsync(t.p, 0, bytes, st);
    return t;
  }
};
}  // namespace

extern "C" pic_status unet_layer_forward(unet_handle* n, int32_t layer, const float* x, float* y, int32_t relu) {
  if (!n || !x || !y || layer < 0 || layer >= kNL) return fail(n, PIC_EINVAL, "unet_layer_forward: bad argument");
  const Layer& L = n->L[layer];
  const int lev = L.def.level;
  const Vol& v = n->vol[lev];
  cudaStream_t st = n->stream;
  Scratch sc;
  Tensor tin = sc.tensor(v, L.cin, lev, st), tout = sc.tensor(v, L.def.cout, lev, st);
  if (!tin.p || !tout.p) return fail(n, PIC_ENOMEM, "unet_layer_forward: scratch");
  const long long nv = (long long)v.D * v.H * v.W;
  ULAUNCH(grid_for(nv), 256, 0, st, k_pack_dense)(v, L.def.cin, L.cin / 8, x, tin.p);
  conv(n, layer, false, tin, nullptr, tout, nullptr, nullptr, nullptr, relu != 0, st);
  ULAUNCH(grid_for(nv), 256, 0, st, k_unpack_dense)(v, L.def.cout, tout.p, y);
  if (cudaGetLastError() != cudaSuccess) return fail(n, PIC_ECUDA, "unet_layer_forward: launch failed");
  return check_err(n);
}

extern "C" pic_status unet_layer_backward(unet_handle* n, int32_t layer, const float* x, const float* dz, float* dx,
                                          float* dw_host, int64_t ndw) {
  if (!n || !x || !dz || !dw_host || layer < 0 || layer >= kNL)
    return fail(n, PIC_EINVAL, "unet_layer_backward: bad argument");
  Layer& L = n->L[layer];
  if (ndw != 27ll * L.def.cin * L.def.cout)
    return fail(n, PIC_EINVAL, "unet_layer_backward: dw needs %lld values", 27ll * L.def.cin * L.def.cout);
  const int lev = L.def.level;
  const Vol& v = n->vol[lev];
  cudaStream_t st = n->stream;
  Scratch sc;
  Tensor tin = sc.tensor(v, L.cin, lev, st), tdz = sc.tensor(v, L.def.cout, lev, st);
  Tensor tdx = sc.tensor(v, L.cin, lev, st);
  if (!tin.p || !tdz.p || !tdx.p) return fail(n, PIC_ENOMEM, "unet_layer_backward: scratch");
  const long long nv = (long long)v.D * v.H * v.W;
  ULAUNCH(grid_for(nv), 256, 0, st, k_pack_dense)(v, L.def.cin, L.cin / 8, x, tin.p);
  ULAUNCH(grid_for(nv), 256, 0, st, k_pack_dense)(v, L.def.cout, L.def.cout / 8, dz, tdz.p);
  if (cudaMemsetAsync(L.g, 0, sizeof(float) * L.nw(), st) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet_layer_backward: memset failed");
  wgrad(n, layer, tin, nullptr, tdz, st);
  conv(n, layer, true, tdz, nullptr, tdx, nullptr, nullptr, nullptr, false, st);
  if (dx) ULAUNCH(grid_for(nv), 256, 0, st, k_unpack_dense)(v, L.def.cin, tdx.p, dx);
  std::vector<float> g(L.nw());
  if (cudaMemcpyAsync(g.data(), L.g, sizeof(float) * L.nw(), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet_layer_backward: copy failed");
  pic_status ps = check_err(n);
  if (ps != PIC_OK) return ps;
  store_to_host(L.def, L.cin, g.data(), dw_host);
  return PIC_OK;
}

extern "C" pic_status unet_train_step_residual(unet_handle* n, const float* x, float lr, double* loss) {
  if (!n || !x || !(lr >= 0.f)) return fail(n, PIC_EINVAL, "unet_train_step_residual: bad argument");
  cudaStream_t st = n->stream;
  const Vol& v = n->vol[0];
  const long long nv = (long long)v.D * v.H * v.W;
  cudaError_t e = forward(n, x, n->y, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->red + 3, 0, sizeof(double), st);
  if (e != cudaSuccess) return fail(n, PIC_ECUDA, "unet_train_step_residual: %s", cudaGetErrorString(e));
  float* ebuf = n->xin;  // scratch (the warm start's input buffer)
  ULAUNCH(grid_for(nv), 256, 0, st, k_resid_e)(v, x, n->y, ebuf, n->red + 3);
  ULAUNCH(grid_for(nv), 256, 0, st, k_resid_dy)(v, ebuf, 1.0 / ((double)(v.D - 1) * v.H * v.W), n->dy, n->red + 3);
  e = backward(n, n->dy, nullptr, v.D, st);
  if (e != cudaSuccess) return fail(n, PIC_ECUDA, "unet_train_step_residual: %s", cudaGetErrorString(e));
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
  ULAUNCH(grid_for(n->n_store), 256, 0, st, k_adam)(n->wbuf, n->wbuf + n->n_store, n->wbuf + 2 * n->n_store,
                                                    n->wbuf + 3 * n->n_store, n->n_store, lr, b1, b2, 1e-8f, c1, c2);
  rebuild_images(n, st);
  n->have_forward = false;
  if (loss && cudaMemcpyAsync(loss, n->red + 3, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet_train_step_residual: loss read failed");
  return check_err(n);
}

extern "C" pic_status unet_make_sample(unet_handle* n, const double* pn, const double* po, float* x, float* t,
                                       double* s_out) {
  if (!n || !pn || !po || !x || !t) return fail(n, PIC_EINVAL, "unet_make_sample: null argument");
  const Vol& v = n->vol[0];
  const long long nv = (long long)v.D * v.H * v.W;
  cudaStream_t st = n->stream;
  if (cudaMemsetAsync(n->red + 1, 0, sizeof(double), st) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet_make_sample: memset failed");
  ULAUNCH(grid_for(nv), 256, 0, st, k_sample_delta)(v, pn, po, x, t, n->red + 1);
  ULAUNCH(grid_for(nv), 256, 0, st, k_sample_scale)(v, n->red + 1, (double)(v.D - 1) * v.H * v.W, x, x + nv, t,
                                                    n->red + 2);
  if (s_out && cudaMemcpyAsync(s_out, n->red + 2, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet_make_sample: read failed");
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail(n, PIC_ECUDA, "unet_make_sample: CUDA error");
  return PIC_OK;
}
