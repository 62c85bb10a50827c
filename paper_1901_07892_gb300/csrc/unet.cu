// Learned coarse-grid correction for the pressure multigrid: a small 3-D
// U-Net (three levels of widths c0/c1/c2, two 3x3x3 convolutions + ReLU per
// level, 2x2x2 average pooling, nearest up-sampling with skip concatenation,
// 1x1x1 head to one channel), BF16 activations and weights, float32
// accumulation on the tensor cores, float32 master weights trained with Adam
// by this file's own forward and backward kernels.  The paper has no learned
// component; the network extends its pressure solve.
//
// Layout: activations [Z][Y][X][C] bf16, C a multiple of 16 (the 3 input
// channels are padded to 16).  A 3x3x3 convolution is an implicit GEMM:
// rows = voxels, K = 27 taps x C_in, N = C_out, computed on the tcgen05
// tensor cores with the accumulator in tensor memory (k_conv3_tc below).
// Forward weights are stored [tap][C_out][C_in] (C_in contiguous: the B
// operand's rows); the input-gradient pass is the same kernel with the
// flipped, transposed weights [26 - tap][C_in][C_out].  Weight gradients are
// float32 reductions over voxels on the CUDA cores.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace wsi {

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ unsigned int ld32(const bf16* p) { return *reinterpret_cast<const unsigned int*>(p); }

// input of a convolution: channels [0, C0) from in0 (read at half resolution
// when up0: nearest up-sampling), channels [C0, C0 + C1) from in1
struct ConvIn {
  const bf16* in0;
  int C0, up0;
  const bf16* in1;
  int C1;
};

// 32-bit load of channels (c, c+1) of the concatenated input at voxel
// (x, y, z) of the output grid (Z, Y, X); zero outside the grid
__device__ __forceinline__ unsigned int in_pair(const ConvIn& a, int Z, int Y, int X, int z, int y, int x, int c) {
  if (z < 0 || z >= Z || y < 0 || y >= Y || x < 0 || x >= X) return 0u;
  if (c < a.C0) {
    if (a.up0) {
      int Yh = Y >> 1, Xh = X >> 1;
      size_t v = ((size_t)(z >> 1) * Yh + (y >> 1)) * Xh + (x >> 1);
      return ld32(a.in0 + v * a.C0 + c);
    }
    size_t v = ((size_t)z * Y + y) * X + x;
    return ld32(a.in0 + v * a.C0 + c);
  }
  size_t v = ((size_t)z * Y + y) * X + x;
  return ld32(a.in1 + v * a.C1 + (c - a.C0));
}

// ------------------------------------------------------------------ conv on tcgen05
// The same implicit GEMM on the fifth-generation tensor cores: one CTA (4
// warps) computes 128 consecutive voxels (M = 128) times all output channels
// (N = Cout) into a float32 accumulator in tensor memory; K = 27 taps x C_in
// runs in chunks of 16 channels, one tcgen05.mma (kind::f16, bf16 inputs) per
// chunk.  Every thread gathers its voxel's 16 channels of the chunk (zero
// outside the grid: the convolution's padding) and the first N threads the
// weights' rows into this CTA's shared memory, in the K-major layout without
// swizzling (core matrices of 8 rows x 16 bytes; neighbours along K 128
// bytes apart, along M/N 256 bytes apart).  Two stages alternate: while the
// tensor core works on one, the threads fill the other; the MMA's completion
// is signalled to an mbarrier by tcgen05.commit.  The epilogue reads the
// accumulator rows back with tcgen05.ld (warp w owns lanes 32w..32w+31), adds
// the bias, applies the ReLU and stores bf16.  Every mbarrier wait is
// bounded: on expiry the kernel sets *err, skips the epilogue and still
// frees its tensor memory.
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: float32 accumulator, bf16 A and B,
// both K-major, shape M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    __nanosleep(64);
  }
  return false;
}

// byte offset of element (row r, channel k in 0..15) in a K-major tile
__device__ __forceinline__ int tile_off(int r, int k) { return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

}  // namespace tc

// 16 channels (cb .. cb+15) of the concatenated input at voxel (x, y, z) of
// the output grid, as two 16-byte words; zero outside the grid
__device__ __forceinline__ void in16(const ConvIn& a, int Z, int Y, int X, int z, int y, int x, int cb, uint4& lo,
                                     uint4& hi) {
  lo = make_uint4(0u, 0u, 0u, 0u);
  hi = lo;
  if (z < 0 || z >= Z || y < 0 || y >= Y || x < 0 || x >= X) return;
  const bf16* p;
  if (cb < a.C0) {
    if (a.up0) {
      const int Yh = Y >> 1, Xh = X >> 1;
      p = a.in0 + (((size_t)(z >> 1) * Yh + (y >> 1)) * Xh + (x >> 1)) * a.C0 + cb;
    } else {
      p = a.in0 + (((size_t)z * Y + y) * X + x) * a.C0 + cb;
    }
  } else {
    p = a.in1 + (((size_t)z * Y + y) * X + x) * a.C1 + (cb - a.C0);
  }
  lo = *reinterpret_cast<const uint4*>(p);
  hi = *reinterpret_cast<const uint4*>(p + 8);
}

template <int N>
__global__ void __launch_bounds__(128) k_conv3_tc(ConvIn a, const bf16* __restrict__ W, const float* __restrict__ bias,
                                                  bf16* out, int Z, int Y, int X, int relu, int* err) {
  constexpr int A_BYTES = 128 * 32, B_BYTES = N * 32, STAGE = A_BYTES + B_BYTES;
  constexpr int TM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  __shared__ __align__(1024) unsigned char sm[2 * STAGE];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Cin = a.C0 + a.C1;
  const size_t V = (size_t)Z * Y * X;
  const size_t v = (size_t)blockIdx.x * 128 + tid;  // this thread's voxel (row)
  const bool vok = v < V;
  const int x = vok ? (int)(v % X) : 0, y = vok ? (int)((v / X) % Y) : 0, z = vok ? (int)(v / ((size_t)X * Y)) : 0;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(&tmem_slot)),
                 "r"(TM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const int chunks_per_tap = Cin / 16, nchunk = 27 * chunks_per_tap;
  constexpr uint32_t IDESC = tc::instr_desc(128, N);
  bool ok = true;
  for (int c = 0; c < nchunk && ok; ++c) {
    const int s = c & 1;
    if (c >= 2) ok = tc::mbar_wait(tc::saddr(&mbar[s]), ((c - 2) >> 1) & 1);  // stage s free again
    if (!ok) break;
    const int tap = c / chunks_per_tap, cb = (c - tap * chunks_per_tap) * 16;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    unsigned char* As = sm + s * STAGE;
    unsigned char* Bs = As + A_BYTES;
    uint4 lo, hi;
    if (vok) {
      in16(a, Z, Y, X, z + dz, y + dy, x + dx, cb, lo, hi);
    } else {
      lo = make_uint4(0u, 0u, 0u, 0u);
      hi = lo;
    }
    *reinterpret_cast<uint4*>(As + tc::tile_off(tid, 0)) = lo;
    *reinterpret_cast<uint4*>(As + tc::tile_off(tid, 8)) = hi;
    if (tid < N) {
      const bf16* wr = W + ((size_t)tap * N + tid) * Cin + cb;
      *reinterpret_cast<uint4*>(Bs + tc::tile_off(tid, 0)) = *reinterpret_cast<const uint4*>(wr);
      *reinterpret_cast<uint4*>(Bs + tc::tile_off(tid, 8)) = *reinterpret_cast<const uint4*>(wr + 8);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t ad = tc::smem_desc(tc::saddr(As), 128, 256), bd = tc::smem_desc(tc::saddr(Bs), 128, 256);
      const uint32_t acc = c > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          tc::saddr(&mbar[s])));
    }
  }
  // every issued chunk has completed once the last two commits have arrived
  if (ok) {
    for (int c = (nchunk >= 2 ? nchunk - 2 : 0); c < nchunk && ok; ++c)
      ok = tc::mbar_wait(tc::saddr(&mbar[c & 1]), (c >> 1) & 1);
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const size_t vr = (size_t)blockIdx.x * 128 + 32 * warp + (tid & 31);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (vr < V) {
        __nv_bfloat162 o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float v0 = __uint_as_float(r[2 * q]) + (bias ? bias[c0 + 2 * q] : 0.f);
          float v1 = __uint_as_float(r[2 * q + 1]) + (bias ? bias[c0 + 2 * q + 1] : 0.f);
          if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          o[q] = __floats2bfloat162_rn(v0, v1);
        }
        uint4* dst = reinterpret_cast<uint4*>(out + vr * N + c0);
        dst[0] = *reinterpret_cast<uint4*>(&o[0]);
        dst[1] = *reinterpret_cast<uint4*>(&o[4]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS));
}

static bool conv3_tc(const ConvIn& a, const bf16* W, const float* bias, bf16* out, int Cout, int Z, int Y, int X,
                     bool relu, int* err, cudaStream_t st) {
  const size_t V = (size_t)Z * Y * X;
  dim3 grid((unsigned)((V + 127) / 128));
  switch (Cout) {
    case 16: k_conv3_tc<16><<<grid, 128, 0, st>>>(a, W, bias, out, Z, Y, X, relu, err); break;
    case 32: k_conv3_tc<32><<<grid, 128, 0, st>>>(a, W, bias, out, Z, Y, X, relu, err); break;
    case 48: k_conv3_tc<48><<<grid, 128, 0, st>>>(a, W, bias, out, Z, Y, X, relu, err); break;
    case 64: k_conv3_tc<64><<<grid, 128, 0, st>>>(a, W, bias, out, Z, Y, X, relu, err); break;
    case 80: k_conv3_tc<80><<<grid, 128, 0, st>>>(a, W, bias, out, Z, Y, X, relu, err); break;
    case 96: k_conv3_tc<96><<<grid, 128, 0, st>>>(a, W, bias, out, Z, Y, X, relu, err); break;
    default: return false;
  }
  WSI_COUNT();
  return true;
}

static void conv3(const ConvIn& a, const bf16* W, const float* bias, bf16* out, int Cout, int Z, int Y, int X,
                  bool relu, int* err, cudaStream_t st) {
  // widths are multiples of 16 up to 96 (checked when the network is made)
  if (!conv3_tc(a, W, bias, out, Cout, Z, Y, X, relu, err, st)) cudaMemsetAsync(err, 0xFF, sizeof(int), st);
}

// ------------------------------------------------------------------ elementwise
__global__ void k_pool(const bf16* __restrict__ in, bf16* out, int Z, int Y, int X, int C) {
  // in: (Z, Y, X) fine; out: (Z/2, Y/2, X/2)
  size_t n = (size_t)(Z / 2) * (Y / 2) * (X / 2) * C;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % C);
    size_t v = t / C;
    int x = (int)(v % (X / 2)), y = (int)((v / (X / 2)) % (Y / 2)), z = (int)(v / ((size_t)(X / 2) * (Y / 2)));
    float s = 0.f;
    for (int o = 0; o < 8; ++o) {
      int zz = 2 * z + (o >> 2), yy = 2 * y + ((o >> 1) & 1), xx = 2 * x + (o & 1);
      s += __bfloat162float(in[(((size_t)zz * Y + yy) * X + xx) * C + c]);
    }
    out[t] = __float2bfloat16(s * 0.125f);
  }
}

// d_fine (+)= pool adjoint of d_coarse: each child gets 1/8 of its parent
__global__ void k_pool_bwd(const bf16* __restrict__ dc, bf16* df, int Z, int Y, int X, int C, int accumulate) {
  size_t n = (size_t)Z * Y * X * C;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % C);
    size_t v = t / C;
    int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((size_t)X * Y));
    float g = 0.125f * __bfloat162float(dc[(((size_t)(z >> 1) * (Y >> 1) + (y >> 1)) * (X >> 1) + (x >> 1)) * C + c]);
    if (accumulate) g += __bfloat162float(df[t]);
    df[t] = __float2bfloat16(g);
  }
}

// d_coarse = up-sampling adjoint (sum of the 8 children) of channels
// [0, Cc) of a fine gradient with Ct channels
__global__ void k_up_bwd(const bf16* __restrict__ df, bf16* dc, int Z, int Y, int X, int Ct, int Cc) {
  // Z, Y, X: coarse dims
  size_t n = (size_t)Z * Y * X * Cc;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % Cc);
    size_t v = t / Cc;
    int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((size_t)X * Y));
    float s = 0.f;
    for (int o = 0; o < 8; ++o) {
      int zz = 2 * z + (o >> 2), yy = 2 * y + ((o >> 1) & 1), xx = 2 * x + (o & 1);
      s += __bfloat162float(df[(((size_t)zz * (2 * Y) + yy) * (2 * X) + xx) * Ct + c]);
    }
    dc[t] = __float2bfloat16(s);
  }
}

// d[v][c] = (y[v][c] > 0) ? d : 0, optionally reading d from channels
// [coff, coff + C) of a wider tensor (Ct channels) into a packed one
__global__ void k_relu_mask(const bf16* __restrict__ d, int Ct, int coff, const bf16* __restrict__ y, bf16* out,
                            size_t V, int C) {
  size_t n = V * C;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % C);
    size_t v = t / C;
    float g = __bfloat162float(d[v * Ct + coff + c]);
    out[t] = __bfloat162float(y[t]) > 0.f ? __float2bfloat16(g) : __float2bfloat16(0.f);
  }
}

// dst += src (bf16, same shape), for gradients meeting at a skip connection
__global__ void k_add_from(bf16* dst, const bf16* __restrict__ src, int Cs, int soff, size_t V, int C) {
  size_t n = V * C;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % C);
    size_t v = t / C;
    dst[t] = __float2bfloat16(__bfloat162float(dst[t]) + __bfloat162float(src[v * Cs + soff + c]));
  }
}

// head: out[v] = sum_c w[c] in[v][c] + b
__global__ void k_head(const bf16* __restrict__ in, const float* __restrict__ w, const float* __restrict__ b, float* out,
                       size_t V, int C) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    float s = b[0];
    for (int c = 0; c < C; ++c) s += w[c] * __bfloat162float(in[v * C + c]);
    out[v] = s;
  }
}

// loss 0.5 mean (out - tgt)^2 -> dout, head gradients, input gradient of the head
__global__ void k_head_bwd(const float* __restrict__ out, const float* __restrict__ tgt, const bf16* __restrict__ in,
                           const float* __restrict__ w, size_t V, int C, float* gw, float* gb, bf16* din,
                           double* loss) {
  float lw[16];
  for (int c = 0; c < C; ++c) lw[c] = 0.f;
  float lb = 0.f;
  double ls = 0.0;
  const float invN = 1.0f / (float)V;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
    float e = out[v] - tgt[v];
    ls += 0.5 * (double)e * (double)e;
    float d = e * invN;
    lb += d;
    for (int c = 0; c < C; ++c) {
      lw[c] += d * __bfloat162float(in[v * C + c]);
      din[v * C + c] = __float2bfloat16(w[c] * d);
    }
  }
  for (int c = 0; c < C; ++c) atomicAdd(&gw[c], lw[c]);
  atomicAdd(gb, lb);
  atomicAdd(loss, ls / (double)V);
}

// ------------------------------------------------------------------ weight gradients
// dW[tap][o][c] += sum_v dY[v][o] X_tap[v][c] over a chunk of voxels;
// db[o] += sum_v dY[v][o] (tap 13 blocks only)
__global__ void k_conv_dw(ConvIn a, const bf16* __restrict__ dY, int Cout, int Z, int Y, int X, float* dW, float* db,
                          int chunk) {
  const int tap = blockIdx.y;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int Cin = a.C0 + a.C1;
  const int npairs = Cout * Cin;
  const size_t V = (size_t)Z * Y * X;
  const size_t v0 = (size_t)blockIdx.x * chunk;
  const size_t v1 = v0 + chunk < V ? v0 + chunk : V;
  float acc[24];
  const int per = (npairs + blockDim.x - 1) / blockDim.x;
  for (int q = 0; q < per; ++q) acc[q] = 0.f;
  float bacc = 0.f;
  for (size_t v = v0; v < v1; ++v) {
    int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((size_t)X * Y));
    int zz = z + dz, yy = y + dy, xx = x + dx;
    bool inb = zz >= 0 && zz < Z && yy >= 0 && yy < Y && xx >= 0 && xx < X;
    for (int q = 0; q < per; ++q) {
      int p = threadIdx.x + q * blockDim.x;
      if (p >= npairs) break;
      int o = p / Cin, c = p - o * Cin;
      float gy = __bfloat162float(dY[v * Cout + o]);
      float xv = 0.f;
      if (inb) {
        unsigned int pr = in_pair(a, Z, Y, X, zz, yy, xx, c & ~1);
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&pr);
        xv = (c & 1) ? __high2float(h) : __low2float(h);
      }
      acc[q] += gy * xv;
    }
    if (tap == 13 && threadIdx.x < Cout) bacc += __bfloat162float(dY[v * Cout + threadIdx.x]);
  }
  for (int q = 0; q < per; ++q) {
    int p = threadIdx.x + q * blockDim.x;
    if (p < npairs) {
      int o = p / Cin, c = p - o * Cin;
      atomicAdd(&dW[((size_t)tap * Cout + o) * Cin + c], acc[q]);
    }
  }
  if (tap == 13 && threadIdx.x < Cout) atomicAdd(&db[threadIdx.x], bacc);
}

// ------------------------------------------------------------------ Adam + weight packing
__global__ void k_adam(float* w, const float* __restrict__ g, float* m, float* v, size_t n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    float gt = g[t];
    float mt = b1 * m[t] + (1.f - b1) * gt;
    float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  }
}

// forward weights [tap][o][c] bf16; input-gradient weights [26-tap][c][o]
__global__ void k_pack(const float* __restrict__ w, bf16* wf, bf16* wb, int Cout, int Cin) {
  size_t n = (size_t)27 * Cout * Cin;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % Cin);
    int o = (int)((t / Cin) % Cout);
    int tap = (int)(t / ((size_t)Cin * Cout));
    bf16 b = __float2bfloat16(w[t]);
    wf[t] = b;
    wb[((size_t)(26 - tap) * Cin + c) * Cout + o] = b;
  }
}

static int nblk(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8)); }

// ------------------------------------------------------------------ network object
struct ConvLayer {
  int Cout, C0, C1, up0;  // input = concat(up?(in0: C0), in1: C1)
  size_t woff, boff;      // offsets into the float32 parameter vector
  bf16 *wf = nullptr, *wb = nullptr;
};

struct UNetImpl {
  int Z, Y, X, c0, c1, c2;
  std::vector<ConvLayer> L;  // a1 a2 b1 b2 c1 c2 ub1 ub2 ua1 ua2
  size_t headw, headb, nparam;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  // activations
  bf16 *x = nullptr, *a1 = nullptr, *a2 = nullptr, *pa = nullptr, *b1 = nullptr, *b2 = nullptr, *pb = nullptr,
       *cc1 = nullptr, *cc2 = nullptr, *ub1 = nullptr, *ub2 = nullptr, *ua1 = nullptr, *ua2 = nullptr;
  // gradients (bf16 scratch)
  bf16 *g0 = nullptr, *g1 = nullptr, *g2 = nullptr, *gA = nullptr, *gB = nullptr;
  float *out = nullptr, *tgt = nullptr;
  double* loss = nullptr;
  int* tcerr = nullptr;  // set by a tensor-core convolution whose wait ran out
  int step = 0;
  std::vector<void*> allocs;
};


static bf16* balloc(UNetImpl& u, size_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(bf16)) != cudaSuccess) return nullptr;
  cudaMemset(p, 0, std::max<size_t>(n, 1) * sizeof(bf16));
  u.allocs.push_back(p);
  return (bf16*)p;
}
static float* falloc(UNetImpl& u, size_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(float)) != cudaSuccess) return nullptr;
  cudaMemset(p, 0, std::max<size_t>(n, 1) * sizeof(float));
  u.allocs.push_back(p);
  return (float*)p;
}

UNetImpl* unet_create(int Z, int Y, int X, int c0, int c1, int c2) {
  if (Z % 4 || Y % 4 || X % 4 || c0 % 16 || c1 % 16 || c2 % 16 || c0 > 16 || c1 > 32 || c2 > 64) return nullptr;
  UNetImpl* u = new UNetImpl();
  u->Z = Z;
  u->Y = Y;
  u->X = X;
  u->c0 = c0;
  u->c1 = c1;
  u->c2 = c2;
  // (Cout, C0, C1, up0) of a1 a2 b1 b2 c1 c2 ub1 ub2 ua1 ua2
  const int spec[10][4] = {{c0, 16, 0, 0}, {c0, c0, 0, 0}, {c1, c0, 0, 0}, {c1, c1, 0, 0}, {c2, c1, 0, 0},
                           {c2, c2, 0, 0}, {c1, c2, c1, 1}, {c1, c1, 0, 0}, {c0, c1, c0, 1}, {c0, c0, 0, 0}};
  size_t off = 0;
  for (int l = 0; l < 10; ++l) {
    ConvLayer L;
    L.Cout = spec[l][0];
    L.C0 = spec[l][1];
    L.C1 = spec[l][2];
    L.up0 = spec[l][3];
    L.woff = off;
    off += (size_t)27 * L.Cout * (L.C0 + L.C1);
    L.boff = off;
    off += L.Cout;
    u->L.push_back(L);
  }
  u->headw = off;
  off += c0;
  u->headb = off;
  off += 1;
  u->nparam = off;
  bool ok = true;
  u->w = falloc(*u, off);
  u->g = falloc(*u, off);
  u->m = falloc(*u, off);
  u->v = falloc(*u, off);
  for (auto& L : u->L) {
    size_t n = (size_t)27 * L.Cout * (L.C0 + L.C1);
    L.wf = balloc(*u, n);
    L.wb = balloc(*u, n);
    ok &= L.wf && L.wb;
  }
  size_t V = (size_t)Z * Y * X, V2 = V / 8, V4 = V / 64;
  u->x = balloc(*u, V * 16);
  u->a1 = balloc(*u, V * c0);
  u->a2 = balloc(*u, V * c0);
  u->pa = balloc(*u, V2 * c0);
  u->b1 = balloc(*u, V2 * c1);
  u->b2 = balloc(*u, V2 * c1);
  u->pb = balloc(*u, V4 * c1);
  u->cc1 = balloc(*u, V4 * c2);
  u->cc2 = balloc(*u, V4 * c2);
  u->ub1 = balloc(*u, V2 * c1);
  u->ub2 = balloc(*u, V2 * c1);
  u->ua1 = balloc(*u, V * c0);
  u->ua2 = balloc(*u, V * c0);
  size_t gsz = std::max(V * (c0 + c1), V2 * (c1 + c2));
  u->g0 = balloc(*u, gsz);
  u->g1 = balloc(*u, gsz);
  u->g2 = balloc(*u, gsz);
  u->gA = balloc(*u, V * c0);   // skip gradient of a2
  u->gB = balloc(*u, V2 * c1);  // skip gradient of b2
  u->out = falloc(*u, V);
  u->tgt = falloc(*u, V);
  void* lp = nullptr;
  ok &= cudaMalloc(&lp, sizeof(double)) == cudaSuccess;
  u->loss = (double*)lp;
  u->allocs.push_back(lp);
  u->tcerr = (int*)falloc(*u, 1);
  ok &= u->w && u->g && u->m && u->v && u->x && u->ua2 && u->g2 && u->gB && u->out && u->tgt && u->tcerr;
  if (!ok) {
    unet_destroy(u);
    return nullptr;
  }
  return u;
}

void unet_destroy(UNetImpl* u) {
  if (!u) return;
  for (void* p : u->allocs) cudaFree(p);
  delete u;
}

void unet_pack(UNetImpl* u, cudaStream_t st) {
  for (auto& L : u->L) {
    size_t n = (size_t)27 * L.Cout * (L.C0 + L.C1);
    { k_pack<<<nblk(n), 256, 0, st>>>(u->w + L.woff, L.wf, L.wb, L.Cout, L.C0 + L.C1); WSI_COUNT(); }
  }
}

// forward from u->x (bf16 [V][16]) to u->out (float [V])
void unet_forward(UNetImpl* u, cudaStream_t st) {
  const int Z = u->Z, Y = u->Y, X = u->X, c0 = u->c0, c1 = u->c1, c2 = u->c2;
  auto& L = u->L;
  auto cv = [&](int l, const bf16* in0, const bf16* in1, bf16* out, int z, int y, int x) {
    ConvIn a{in0, L[l].C0, L[l].up0, in1, L[l].C1};
    conv3(a, L[l].wf, u->w + L[l].boff, out, L[l].Cout, z, y, x, true, u->tcerr, st);
  };
  size_t V = (size_t)Z * Y * X;
  cv(0, u->x, nullptr, u->a1, Z, Y, X);
  cv(1, u->a1, nullptr, u->a2, Z, Y, X);
  { k_pool<<<nblk(V / 8 * c0), 256, 0, st>>>(u->a2, u->pa, Z, Y, X, c0); WSI_COUNT(); }
  cv(2, u->pa, nullptr, u->b1, Z / 2, Y / 2, X / 2);
  cv(3, u->b1, nullptr, u->b2, Z / 2, Y / 2, X / 2);
  { k_pool<<<nblk(V / 64 * c1), 256, 0, st>>>(u->b2, u->pb, Z / 2, Y / 2, X / 2, c1); WSI_COUNT(); }
  cv(4, u->pb, nullptr, u->cc1, Z / 4, Y / 4, X / 4);
  cv(5, u->cc1, nullptr, u->cc2, Z / 4, Y / 4, X / 4);
  cv(6, u->cc2, u->b2, u->ub1, Z / 2, Y / 2, X / 2);
  cv(7, u->ub1, nullptr, u->ub2, Z / 2, Y / 2, X / 2);
  cv(8, u->ub2, u->a2, u->ua1, Z, Y, X);
  cv(9, u->ua1, nullptr, u->ua2, Z, Y, X);
  (void)c2;
  { k_head<<<nblk(V), 256, 0, st>>>(u->ua2, u->w + u->headw, u->w + u->headb, u->out, V, c0); WSI_COUNT(); }
}

// One layer's backward: G (gradient of its output, channels [goff, goff+Cout)
// of a tensor with Gt channels) -> weight/bias gradients, and (if dX) the
// input gradient [V][C0 + C1] into dX.
static void layer_bwd(UNetImpl* u, int l, const bf16* in0, const bf16* in1, const bf16* y, const bf16* G, int Gt,
                      int goff, bf16* M, bf16* dX, int z, int yy, int x, cudaStream_t st) {
  ConvLayer& L = u->L[l];
  size_t V = (size_t)z * yy * x;
  { k_relu_mask<<<nblk(V * L.Cout), 256, 0, st>>>(G, Gt, goff, y, M, V, L.Cout); WSI_COUNT(); }
  ConvIn a{in0, L.C0, L.up0, in1, L.C1};
  const int chunk = 1024;
  dim3 grid(cdiv((long long)V, chunk), 27);
  { k_conv_dw<<<grid, 256, 0, st>>>(a, M, L.Cout, z, yy, x, u->g + L.woff, u->g + L.boff, chunk); WSI_COUNT(); }
  if (dX) {
    ConvIn b{M, L.Cout, 0, nullptr, 0};
    conv3(b, L.wb, nullptr, dX, L.C0 + L.C1, z, yy, x, false, u->tcerr, st);
  }
}

// gradients of 0.5 mean((out - tgt)^2) into u->g (zeroed first); loss into u->loss
void unet_backward(UNetImpl* u, cudaStream_t st) {
  const int Z = u->Z, Y = u->Y, X = u->X, c0 = u->c0, c1 = u->c1, c2 = u->c2;
  const size_t V = (size_t)Z * Y * X, V2 = V / 8, V4 = V / 64;
  cudaMemsetAsync(u->g, 0, u->nparam * sizeof(float), st);
  cudaMemsetAsync(u->loss, 0, sizeof(double), st);
  { k_head_bwd<<<nblk(V), 256, 0, st>>>(u->out, u->tgt, u->ua2, u->w + u->headw, V, c0, u->g + u->headw,
                                        u->g + u->headb, u->g0, u->loss); WSI_COUNT(); }
  // full resolution decoder
  layer_bwd(u, 9, u->ua1, nullptr, u->ua2, u->g0, c0, 0, u->g1, u->g2, Z, Y, X, st);           // d ua1 -> g2
  layer_bwd(u, 8, u->ub2, u->a2, u->ua1, u->g2, c0, 0, u->g1, u->g0, Z, Y, X, st);             // d [up(ub2), a2] -> g0
  // skip gradient of a2: gA = g0[:, c1:] (its ReLU mask is applied with the
  // pooled-path gradient, in layer a2's backward)
  cudaMemsetAsync(u->gA, 0, V * c0 * sizeof(bf16), st);
  { k_add_from<<<nblk(V * c0), 256, 0, st>>>(u->gA, u->g0, c1 + c0, c1, V, c0); WSI_COUNT(); }
  { k_up_bwd<<<nblk(V2 * c1), 256, 0, st>>>(u->g0, u->g2, Z / 2, Y / 2, X / 2, c1 + c0, c1); WSI_COUNT(); }  // d ub2
  // half resolution decoder
  layer_bwd(u, 7, u->ub1, nullptr, u->ub2, u->g2, c1, 0, u->g1, u->g0, Z / 2, Y / 2, X / 2, st);  // d ub1 -> g0
  layer_bwd(u, 6, u->cc2, u->b2, u->ub1, u->g0, c1, 0, u->g1, u->g2, Z / 2, Y / 2, X / 2, st);    // d [up(cc2), b2] -> g2
  cudaMemsetAsync(u->gB, 0, V2 * c1 * sizeof(bf16), st);
  { k_add_from<<<nblk(V2 * c1), 256, 0, st>>>(u->gB, u->g2, c2 + c1, c2, V2, c1); WSI_COUNT(); }
  { k_up_bwd<<<nblk(V4 * c2), 256, 0, st>>>(u->g2, u->g0, Z / 4, Y / 4, X / 4, c2 + c1, c2); WSI_COUNT(); }  // d cc2
  // bottom
  layer_bwd(u, 5, u->cc1, nullptr, u->cc2, u->g0, c2, 0, u->g1, u->g2, Z / 4, Y / 4, X / 4, st);  // d cc1 -> g2
  layer_bwd(u, 4, u->pb, nullptr, u->cc1, u->g2, c2, 0, u->g1, u->g0, Z / 4, Y / 4, X / 4, st);   // d pb -> g0
  { k_pool_bwd<<<nblk(V2 * c1), 256, 0, st>>>(u->g0, u->gB, Z / 2, Y / 2, X / 2, c1, 1); WSI_COUNT(); }  // d b2
  // half resolution encoder
  layer_bwd(u, 3, u->b1, nullptr, u->b2, u->gB, c1, 0, u->g1, u->g2, Z / 2, Y / 2, X / 2, st);    // d b1 -> g2
  layer_bwd(u, 2, u->pa, nullptr, u->b1, u->g2, c1, 0, u->g1, u->g0, Z / 2, Y / 2, X / 2, st);    // d pa -> g0
  { k_pool_bwd<<<nblk(V * c0), 256, 0, st>>>(u->g0, u->gA, Z, Y, X, c0, 1); WSI_COUNT(); }        // d a2
  // full resolution encoder
  layer_bwd(u, 1, u->a1, nullptr, u->a2, u->gA, c0, 0, u->g1, u->g2, Z, Y, X, st);                // d a1 -> g2
  layer_bwd(u, 0, u->x, nullptr, u->a1, u->g2, c0, 0, u->g1, nullptr, Z, Y, X, st);
}

// float [V][3] -> the network's bf16 [V][16] input (channels 3..15 zero)
__global__ void k_input3(const float* __restrict__ x3, bf16* x, size_t V) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x)
    for (int c = 0; c < 16; ++c) x[v * 16 + c] = __float2bfloat16(c < 3 ? x3[v * 3 + c] : 0.f);
}

void unet_set_input3(UNetImpl* u, const float* x3, cudaStream_t st) {
  size_t V = (size_t)u->Z * u->Y * u->X;
  { k_input3<<<nblk(V), 256, 0, st>>>(x3, u->x, V); WSI_COUNT(); }
}

int unet_dim(const UNetImpl* u, int axis) { return axis == 0 ? u->Z : (axis == 1 ? u->Y : u->X); }
size_t unet_nparam(const UNetImpl* u) { return u->nparam; }
float* unet_params(UNetImpl* u) { return u->w; }
float* unet_grads(UNetImpl* u) { return u->g; }
__nv_bfloat16* unet_input(UNetImpl* u) { return u->x; }
float* unet_output(UNetImpl* u) { return u->out; }
float* unet_target(UNetImpl* u) { return u->tgt; }
double* unet_loss(UNetImpl* u) { return u->loss; }
float* unet_moment(UNetImpl* u, int which) { return which == 0 ? u->m : u->v; }
int* unet_step_count(UNetImpl* u) { return &u->step; }
bool unet_take_error(UNetImpl* u) {
  int h = 0;
  if (cudaMemcpy(&h, u->tcerr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return true;
  if (h) cudaMemset(u->tcerr, 0, sizeof(int));
  return h != 0;
}

int unet_width(const UNetImpl* u, int level) { return level == 0 ? u->c0 : (level == 1 ? u->c1 : u->c2); }

void unet_adam(UNetImpl* u, double lr, cudaStream_t st) {
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
  { k_adam<<<nblk(u->nparam), 256, 0, st>>>(u->w, u->g, u->m, u->v, u->nparam, (float)lr, b1, b2, c1, c2, 1e-8f); WSI_COUNT(); }
  unet_pack(u, st);
}

}  // namespace wsi
