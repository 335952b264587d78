// spod_blocks.cu -- the SPOD front end of pyLOM (arXiv 2405.15529, Sec. 2.3
// and Alg. 6): the snapshots D (N points x T instants) are cut into nBlks
// blocks of npwin instants overlapping by nolap, every point's block is
// multiplied by the Hamming window w_j = 0.54 - 0.46 cos(2 pi j/(npwin-1)),
// transformed, divided by mean(w) npwin, and the one-sided spectrum
// (k = 0 .. floor(npwin/2), all entries but the first and last doubled, as
// Alg. 6 writes it) is gathered per frequency into Q_f (N x nBlks), scaled
// by 1/sqrt(nBlks): the matrices whose SVDs the batched kernel computes.
//
// For npwin <= 64 the transform runs on the tensor cores (below).  Larger
// windows take the direct form: one thread per (point, block), the npwin
// windowed samples of its point staged in shared memory (column per thread,
// conflict-free), every frequency a direct transform over them with the
// window and the twiddle factors read from shared tables.  Reads of D are coalesced across the points of a block; each Q_f
// column is written coalesced.  FP32 arithmetic (the bins are complex64),
// the temporal mean and the tables in binary64.
#include <math.h>

#include "kernels.h"
#include "tc05.cuh"

namespace pylom {

constexpr int kSpodThreads = 128;
constexpr int64_t kSpodMaxWin = 512;

// tables (float): window[npwin], cos[npwin], sin[npwin] of 2 pi m / npwin
__global__ void spod_tables_kernel(float* tab, int64_t npwin) {
  for (int64_t m = threadIdx.x; m < npwin; m += blockDim.x) {
    const double a = 2.0 * M_PI * (double)m / (double)npwin;
    tab[m] = (float)(0.54 - 0.46 * cos(2.0 * M_PI * (double)m / (double)(npwin - 1)));
    tab[npwin + m] = (float)cos(a);
    tab[2 * npwin + m] = (float)sin(a);
  }
}

// temporal mean of every point, binary64 accumulation (one thread per point)
__global__ void spod_mean_kernel(const double* D, int64_t N, int64_t T, int64_t ldd, double* mean) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  double s = 0.0;
  for (int64_t t = 0; t < T; ++t) s += D[p + t * ldd];
  mean[p] = s / (double)T;
}

// binary32 input: chunks of kMeanChunk instants are summed in binary32 with
// an error-free transformation (Knuth's TwoSum: the rounding error of every
// addition is carried in c), and only the pair (s, c) of each chunk is
// added in binary64.  The chunk sum is then exact up to a second-order term
// (about (kMeanChunk eps32)^2 of the sum of magnitudes, 4e-12 here), while
// the binary64 instruction count drops kMeanChunk-fold: on this GPU the
// binary64 pipe, not the memory, set the time of a per-sample binary64 sum.
constexpr int kMeanChunk = 32;
__global__ void spod_mean_f32_kernel(const float* D, int64_t N, int64_t T, int64_t ldd, double* mean) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const float* col = D + p;
  double acc = 0.0;
  int64_t t = 0;
  for (; t + kMeanChunk <= T; t += kMeanChunk) {
    float x[kMeanChunk];
#pragma unroll
    for (int j = 0; j < kMeanChunk; ++j) x[j] = col[(t + j) * ldd];
    float s, c;
    sum32_compensated(x, s, c);
    acc += (double)s + (double)c;
  }
  for (; t < T; ++t) acc += (double)col[t * ldd];
  mean[p] = acc / (double)T;
}

// grid (ceil(N / kSpodThreads), nBlks); dynamic shared memory:
// npwin x kSpodThreads samples + 3 npwin table entries (floats)
template <typename TD>
__global__ void __launch_bounds__(kSpodThreads) spod_blocks_kernel(const TD* D, int64_t N, int64_t ldd,
                                                                  const double* mean, const float* tab,
                                                                  int64_t npwin, int64_t nolap, int64_t nblks,
                                                                  float2* Q, int64_t ldq, float scale) {
  extern __shared__ float ssm[];
  float* xs = ssm;                              // [j][thread]
  float* sw = xs + npwin * kSpodThreads;        // window
  float* sc = sw + npwin;                       // cos(2 pi m / n)
  float* ss = sc + npwin;                       // sin(2 pi m / n)
  const int tid = threadIdx.x;
  for (int64_t m = tid; m < 3 * npwin; m += kSpodThreads) sw[m] = tab[m];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * kSpodThreads + tid;
  const int64_t b = blockIdx.y;
  const int64_t i0 = b * (npwin - nolap);
  const bool live = p < N;
  const double mu = (live && mean) ? mean[p] : 0.0;
  const float muf = (float)mu;
  for (int64_t j = 0; j < npwin; ++j) {
    float x = 0.f;
    if (live) {
      // float input: FP32 subtraction (FP64 arithmetic is slow on this part);
      // double input: the difference in binary64, then rounded
      if constexpr (sizeof(TD) == 4) x = D[p + (i0 + j) * ldd] - muf;
      else x = (float)(D[p + (i0 + j) * ldd] - mu);
    }
    xs[j * kSpodThreads + tid] = x * sw[j];
  }
  // (own column only: no barrier needed before reading it back)
  const int64_t nfreq = npwin / 2 + 1;
  for (int64_t k = 0; k < nfreq; ++k) {
    float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
    int64_t m = 0;   // (k j) mod npwin, advanced by k per sample
    int64_t j = 0;
    for (; j + 1 < npwin; j += 2) {
      const float x0 = xs[j * kSpodThreads + tid];
      re0 = fmaf(x0, sc[m], re0);
      im0 = fmaf(-x0, ss[m], im0);
      m += k;
      if (m >= npwin) m -= npwin;
      const float x1 = xs[(j + 1) * kSpodThreads + tid];
      re1 = fmaf(x1, sc[m], re1);
      im1 = fmaf(-x1, ss[m], im1);
      m += k;
      if (m >= npwin) m -= npwin;
    }
    if (j < npwin) {
      const float x0 = xs[j * kSpodThreads + tid];
      re0 = fmaf(x0, sc[m], re0);
      im0 = fmaf(-x0, ss[m], im0);
    }
    const float c = (k > 0 && k < nfreq - 1) ? 2.f * scale : scale;
    if (live) Q[(k * nblks + b) * ldq + p] = make_float2((re0 + re1) * c, (im0 + im1) * c);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form (npwin <= 64): the transform of a tile of 128 points is a
// dense contraction Q_tile (128 x 2 nfreq) = X_tile (128 x npwin) F, with the
// window, the one-sided doubling and the scaling folded into F:
//   F[j][k]        =  c_k w_j cos(2 pi k j / npwin) / (mean(w) npwin sqrt(nBlks))
//   F[j][kFIm + k] = -c_k w_j sin(2 pi k j / npwin) / (mean(w) npwin sqrt(nBlks))
// (the imaginary parts at a fixed column offset, so the epilogue indexes
// its registers statically).  3xTF32 on tcgen05 (hi*hi into one TMEM
// accumulator, hi*lo + lo*hi into another), K = npwin padded to 64, N = kFN.
// F is built once in binary64 (split hi/lo, core-matrix layout) by a setup
// kernel; every CTA copies it to shared memory and loops over all blocks of
// its 128 points.
// ---------------------------------------------------------------------------
constexpr int kFK = 64;          // K (samples), padded
constexpr int kFN = 80;          // N: real parts in columns 0..32, imaginary parts in kFIm..kFIm+32
constexpr int kFIm = kFN / 2;
constexpr int kFThreads = 128;
constexpr int kFA = 128 * kFK * 4;               // A tile (hi or lo): 32 KB
constexpr int kFB = kFN * kFK * 4;               // F (hi or lo): 20 KB
constexpr int kFSmem = 2 * kFA + 2 * kFB;        // 104 KB
constexpr uint32_t kFTmem = 256;                 // 2 x kFN accumulator columns, rounded up

// F in the K-major core-matrix layout, hi then lo (2 x kFB bytes of floats)
__global__ void spod_ftab_kernel(float* Fhl, int64_t npwin, int64_t nblks) {
  const int64_t nfreq = npwin / 2 + 1;
  double wsum = 0.0;
  for (int64_t j = 0; j < npwin; ++j) wsum += 0.54 - 0.46 * cos(2.0 * M_PI * (double)j / (double)(npwin - 1));
  const double scale = 1.0 / (wsum * sqrt((double)nblks));
  for (int idx = threadIdx.x; idx < kFN * kFK; idx += blockDim.x) {
    const int n = idx / kFK, j = idx % kFK;    // F^T row n (output column), K index j
    double v = 0.0;
    const int64_t k = n < kFIm ? n : n - kFIm;
    if (j < npwin && k < nfreq) {
      const double c = (k > 0 && k < nfreq - 1) ? 2.0 : 1.0;
      const double wj = 0.54 - 0.46 * cos(2.0 * M_PI * (double)j / (double)(npwin - 1));
      const double a = 2.0 * M_PI * (double)((k * j) % npwin) / (double)npwin;
      v = c * wj * scale * (n < kFIm ? cos(a) : -sin(a));
    }
    float hi, lo;
    tc05::split_tf32((float)v, hi, lo);
    const uint32_t o = tc05::cm_off(n, j, kFK) / 4;
    Fhl[o] = hi;
    Fhl[kFN * kFK + o] = lo;
  }
}

template <typename TD>
__global__ void __launch_bounds__(kFThreads) spod_dft_tc_kernel(const TD* D, int64_t N, int64_t ldd,
                                                               const double* mean, const float* Fhl,
                                                               int64_t npwin, int64_t nolap, int64_t nblks,
                                                               float2* Q, int64_t ldq, WsHeader* hdr) {
  using namespace tc05;
  extern __shared__ __align__(128) unsigned char fsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t p0 = (int64_t)blockIdx.x * 128;
  // F (hi, lo) into shared memory
  {
    const float4* src = (const float4*)Fhl;
    float4* dst = (float4*)(fsm + 2 * kFA);
    for (int i = tid; i < 2 * kFB / 16; i += kFThreads) dst[i] = src[i];
  }
  if (tid == 0) mbar_init(&mbar, 1);
  if (warp == 0) tmem_alloc(&tmem_base, kFTmem);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  const int64_t p = p0 + tid;     // this thread's point (its row of A and of the result)
  const bool live = p < N;
  const double mu = (live && mean) ? mean[p] : 0.0;
  const float muf = (float)mu;
  const int64_t nfreq = npwin / 2 + 1;
  bool ok = true;
  // FP32 input: the samples of block bb (row p of A: samples i0 .. i0 +
  // npwin - 1, zeros in the K padding) are loaded into registers one block
  // ahead, so their latency overlaps the previous block's MMAs and epilogue
  // (a binary64 block would need twice the registers: it is loaded in place)
  constexpr bool kAhead = sizeof(TD) == 4;
  float xn[kAhead ? kFK : 1];
  auto load_block = [&](int64_t bb) {
    if constexpr (kAhead) {
      const int64_t i0 = bb * (npwin - nolap);
#pragma unroll
      for (int j = 0; j < kFK; ++j) xn[j] = (live && j < npwin) ? (float)D[p + (i0 + j) * ldd] : 0.f;
    }
  };
  load_block(0);
  for (int64_t b = 0; b < nblks && ok; ++b) {
    auto stage = [&](int j, float x) {
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t o = cm_off(tid, j, kFK);
      *(float*)(fsm + o) = hi;
      *(float*)(fsm + kFA + o) = lo;
    };
    if constexpr (kAhead) {
#pragma unroll
      for (int j = 0; j < kFK; ++j) stage(j, (live && j < npwin) ? xn[j] - muf : 0.f);
    } else {
      const int64_t i0 = b * (npwin - nolap);
#pragma unroll 4
      for (int j = 0; j < kFK; ++j) stage(j, (live && j < npwin) ? (float)(D[p + (i0 + j) * ldd] - mu) : 0.f);
    }
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t a_hi = smem_u32(fsm), a_lo = smem_u32(fsm + kFA);
      const uint32_t b_hi = smem_u32(fsm + 2 * kFA), b_lo = smem_u32(fsm + 2 * kFA + kFB);
      const uint32_t sbo = (kFK / 4) * 128, lbo = 128;
      const uint32_t id = idesc_tf32(128, kFN);
      for (int kk = 0; kk < kFK / 8; ++kk) {
        const uint32_t o = (uint32_t)kk * 256;
        mma_tf32(tmem, desc(a_hi + o, lbo, sbo), desc(b_hi + o, lbo, sbo), id, kk > 0);
        mma_tf32(tmem + kFN, desc(a_hi + o, lbo, sbo), desc(b_lo + o, lbo, sbo), id, kk > 0);
        mma_tf32(tmem + kFN, desc(a_lo + o, lbo, sbo), desc(b_hi + o, lbo, sbo), id, true);
      }
      commit(&mbar);
    }
    if (b + 1 < nblks) load_block(b + 1);
    const bool w_ok = mbar_wait(&mbar, phase);
    phase ^= 1u;
    fence_after();
    ok = !__syncthreads_or(!w_ok);
    if (!ok) break;
    // epilogue: row p of the accumulators -> Q_k[p, b] for every frequency k
    const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
    float hh[16], xx[16], re[kFN];
#pragma unroll
    for (int c0 = 0; c0 < kFN; c0 += 16) {
      tmem_ld16(tmem + lanebase + (uint32_t)c0, hh);
      tmem_ld16(tmem + lanebase + (uint32_t)(kFN + c0), xx);
#pragma unroll
      for (int j = 0; j < 16; ++j) re[c0 + j] = hh[j] + xx[j];
    }
    if (live) {
#pragma unroll
      for (int k = 0; k < kFIm; ++k)
        if (k < nfreq) Q[(k * nblks + b) * ldq + p] = make_float2(re[k], re[kFIm + k]);
    }
    fence_before();
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kFTmem);
  if (!ok && tid == 0) raise_status(hdr, PYLOM_ERR_TIMEOUT);
}

// order[i] = the bin with the i-th largest leading energy S[f stride]^2,
// ties by index (one block; nfreq is small)
__global__ void spod_order_kernel(const double* S, int64_t nfreq, int64_t stride, int64_t* order) {
  for (int64_t f = threadIdx.x; f < nfreq; f += blockDim.x) {
    const double e = S[f * stride] * S[f * stride];
    int64_t rank = 0;
    for (int64_t g = 0; g < nfreq; ++g) {
      const double eg = S[g * stride] * S[g * stride];
      rank += (eg > e) || (eg == e && g < f);
    }
    order[rank] = f;
  }
}

}  // namespace pylom

using namespace pylom;

extern "C" pylom_status pylom_spod_shape(int64_t T, int64_t npwin, int64_t nolap, int64_t* nblks,
                                         int64_t* nfreq) {
  set_error_message("");
  if (!nblks || !nfreq) {
    set_error_message("pylom_spod_shape: null pointer");
    return PYLOM_ERR_ARG;
  }
  if (npwin < 2 || npwin > kSpodMaxWin || nolap < 0 || nolap >= npwin || T < npwin) {
    set_error_message("pylom_spod_shape: need 2 <= npwin <= %lld, 0 <= nolap < npwin, T >= npwin",
                      (long long)kSpodMaxWin);
    return PYLOM_ERR_SHAPE;
  }
  *nblks = (T - nolap) / (npwin - nolap);
  *nfreq = npwin / 2 + 1;
  return PYLOM_OK;
}

extern "C" size_t pylom_spod_blocks_workspace_size(int64_t N, int64_t npwin) {
  if (N < 1 || npwin < 2 || npwin > kSpodMaxWin) return 0;
  return sizeof(WsHeader) + align256(sizeof(double) * (size_t)N) + align256(sizeof(float) * 3 * (size_t)npwin) +
         align256(2 * (size_t)kFB);
}

extern "C" pylom_status pylom_spod_blocks(const void* D, int64_t N, int64_t T, int64_t ldd, int dtype,
                                          int64_t npwin, int64_t nolap, int remove_mean, void* Q, int64_t ldq,
                                          double* mean, void* ws, size_t ws_bytes, void* stream) {
  set_error_message("");
  if (!D || !Q || !ws) {
    set_error_message("pylom_spod_blocks: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (dtype != PYLOM_F32 && dtype != PYLOM_F64) {
    set_error_message("pylom_spod_blocks: dtype must be PYLOM_F32 or PYLOM_F64");
    return PYLOM_ERR_ARG;
  }
  int64_t nblks = 0, nfreq = 0;
  pylom_status sst = pylom_spod_shape(T, npwin, nolap, &nblks, &nfreq);
  if (sst != PYLOM_OK) return sst;
  if (N < 1 || ldd < N || ldq < N) {
    set_error_message("pylom_spod_blocks: need N >= 1, ldd >= N, ldq >= N");
    return PYLOM_ERR_SHAPE;
  }
  const size_t need = pylom_spod_blocks_workspace_size(N, npwin);
  if (((uintptr_t)ws & 255) != 0 || ws_bytes < need) {
    set_error_message("pylom_spod_blocks: workspace needs %zu bytes, 256-byte aligned", need);
    return PYLOM_ERR_WORKSPACE;
  }
  if (!device_readable(D, "pylom_spod_blocks", "D", &D)) return PYLOM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  double* mu = (double*)(base + sizeof(WsHeader));
  float* tab = (float*)(base + sizeof(WsHeader) + align256(sizeof(double) * (size_t)N));
  cudaError_t e = cudaMemsetAsync(base, 0, sizeof(WsHeader), st);
  if (e == cudaSuccess) {
    spod_tables_kernel<<<1, 256, 0, st>>>(tab, npwin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && remove_mean) {
    const unsigned mgrid = (unsigned)((N + 255) / 256);
    if (dtype == PYLOM_F32)
      spod_mean_f32_kernel<<<mgrid, 256, 0, st>>>((const float*)D, N, T, ldd, mu);
    else
      spod_mean_kernel<<<mgrid, 256, 0, st>>>((const double*)D, N, T, ldd, mu);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && remove_mean && mean) e = cudaMemcpyAsync(mean, mu, sizeof(double) * (size_t)N,
                                                                    cudaMemcpyDeviceToDevice, st);
  float* Fhl = (float*)((char*)tab + align256(sizeof(float) * 3 * (size_t)npwin));
  if (e == cudaSuccess && npwin <= kFK) {
    // tensor-core path
    spod_ftab_kernel<<<1, 256, 0, st>>>(Fhl, npwin, nblks);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)spod_dft_tc_kernel<float>, kFSmem);
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)spod_dft_tc_kernel<double>, kFSmem);
    if (e == cudaSuccess) {
      const unsigned grid = (unsigned)((N + 127) / 128);
      if (dtype == PYLOM_F32)
        spod_dft_tc_kernel<float><<<grid, kFThreads, kFSmem, st>>>((const float*)D, N, ldd, remove_mean ? mu : nullptr,
                                                                   Fhl, npwin, nolap, nblks, (float2*)Q, ldq,
                                                                   (WsHeader*)base);
      else
        spod_dft_tc_kernel<double><<<grid, kFThreads, kFSmem, st>>>((const double*)D, N, ldd,
                                                                    remove_mean ? mu : nullptr, Fhl, npwin, nolap,
                                                                    nblks, (float2*)Q, ldq, (WsHeader*)base);
      e = cudaGetLastError();
    }
  } else if (e == cudaSuccess) {
    const size_t smem = sizeof(float) * ((size_t)npwin * kSpodThreads + 3 * (size_t)npwin);
    if (smem > 48 * 1024) {
      e = ensure_dyn_smem((const void*)spod_blocks_kernel<float>, smem);
      if (e == cudaSuccess) e = ensure_dyn_smem((const void*)spod_blocks_kernel<double>, smem);
    }
    if (e == cudaSuccess) {
      // scale: 1 / (mean(w) npwin sqrt(nBlks)); sum_j w_j = 0.54 npwin - 0.46 sum_j cos(2 pi j/(npwin-1))
      double wsum = 0.0;
      for (int64_t j = 0; j < npwin; ++j) wsum += 0.54 - 0.46 * cos(2.0 * M_PI * (double)j / (double)(npwin - 1));
      const float scale = (float)(1.0 / (wsum * sqrt((double)nblks)));
      dim3 grid((unsigned)((N + kSpodThreads - 1) / kSpodThreads), (unsigned)nblks);
      if (dtype == PYLOM_F32)
        spod_blocks_kernel<float><<<grid, kSpodThreads, smem, st>>>((const float*)D, N, ldd, remove_mean ? mu : nullptr,
                                                                    tab, npwin, nolap, nblks, (float2*)Q, ldq, scale);
      else
        spod_blocks_kernel<double><<<grid, kSpodThreads, smem, st>>>((const double*)D, N, ldd,
                                                                     remove_mean ? mu : nullptr, tab, npwin, nolap,
                                                                     nblks, (float2*)Q, ldq, scale);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    set_error_message("pylom_spod_blocks: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}

extern "C" pylom_status pylom_spod_order(const double* S, int64_t nfreq, int64_t stride, int64_t* order,
                                         void* stream) {
  set_error_message("");
  if (!S || !order || nfreq < 1 || stride < 1) {
    set_error_message("pylom_spod_order: null pointer, nfreq < 1 or stride < 1");
    return PYLOM_ERR_ARG;
  }
  spod_order_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(S, nfreq, stride, order);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error_message("pylom_spod_order: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}
