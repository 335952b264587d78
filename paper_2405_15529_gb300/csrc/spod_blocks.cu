// spod_blocks.cu -- the SPOD front end of pyLOM (arXiv 2405.15529, Sec. 2.3
// and Alg. 6): the snapshots D (N points x T instants) are cut into nBlks
// blocks of npwin instants overlapping by nolap, every point's block is
// multiplied by the Hamming window w_j = 0.54 - 0.46 cos(2 pi j/(npwin-1)),
// transformed, divided by mean(w) npwin, and the one-sided spectrum
// (k = 0 .. floor(npwin/2), all entries but the first and last doubled, as
// Alg. 6 writes it) is gathered per frequency into Q_f (N x nBlks), scaled
// by 1/sqrt(nBlks): the matrices whose SVDs the batched kernel computes.
//
// One thread per (point, block): the npwin windowed samples of its point
// are staged in shared memory (column per thread, conflict-free), and every
// frequency is a direct transform over them with the window and the
// twiddle factors read from shared tables (any npwin, including the paper's
// 60).  Reads of D are coalesced across the points of a block; each Q_f
// column is written coalesced.  FP32 arithmetic (the bins are complex64),
// the temporal mean and the tables in binary64.
#include <math.h>

#include "kernels.h"

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

template <typename TD>
__global__ void spod_mean_kernel(const TD* D, int64_t N, int64_t T, int64_t ldd, double* mean) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t t = 0; t < T; ++t) s += (double)D[p + t * ldd];
    mean[p] = s / (double)T;
  }
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
  return sizeof(WsHeader) + align256(sizeof(double) * (size_t)N) + align256(sizeof(float) * 3 * (size_t)npwin);
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
    if (dtype == PYLOM_F32)
      spod_mean_kernel<float><<<512, 256, 0, st>>>((const float*)D, N, T, ldd, mu);
    else
      spod_mean_kernel<double><<<512, 256, 0, st>>>((const double*)D, N, T, ldd, mu);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && remove_mean && mean) e = cudaMemcpyAsync(mean, mu, sizeof(double) * (size_t)N,
                                                                    cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    const size_t smem = sizeof(float) * ((size_t)npwin * kSpodThreads + 3 * (size_t)npwin);
    static size_t smem_set = 0;
    if (smem > 48 * 1024 && smem > smem_set) {
      e = cudaFuncSetAttribute(spod_blocks_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(spod_blocks_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) smem_set = smem;
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
