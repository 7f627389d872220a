// Elementwise device helpers of the runtime: precision conversion, the
// isotropic equilibrium intensity, the sec. 3 quadrature of a given field,
// and input scans.  All grid-stride, sized as a multiple of the SM count.
#include <cuda_bf16.h>
#include <math.h>

#include "rt_internal.h"

namespace rtg {

namespace {

constexpr double kPi = 3.14159265358979323846;

int grid_for(long long n, int threads) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  long long want = (n + threads - 1) / threads;
  long long cap = (long long)sms * 8;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

template <typename Real>
__global__ void convert_in_kernel(const double *__restrict__ src, Real *__restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (Real)src[i];
}

template <typename Real>
__global__ void convert_out_kernel(const Real *__restrict__ src, double *__restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

template <typename Real>
__global__ void isotropic_kernel(const double *__restrict__ T, Real *__restrict__ I, int M, long long N) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    double t = T[c];
    Real b = (Real)(t * t * t * t / (4.0 * kPi));
    for (int m = 0; m < M; ++m) I[(long long)m * N + c] = b;
  }
}

// bf16 storage: delta = I / J - 1 with J = E / (4 pi) of the cell (the same
// arithmetic as the step kernel's b16_* helpers in rt_step_pair.cuh).
constexpr float kInv4PiF = float(1.0 / (4.0 * 3.14159265358979323846));

__global__ void encode_b16_kernel(const float *__restrict__ I, const float *__restrict__ E,
                                  unsigned short *__restrict__ out, int M, long long N) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const float J = E[c] * kInv4PiF;
    const float rJ = J > 1e-30f ? 1.0f / J : 0.0f;
    for (int m = 0; m < M; ++m) {
      const long long i = (long long)m * N + c;
      out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(fmaf(I[i], rJ, -1.0f)));
    }
  }
}

__global__ void decode_b16_kernel(const unsigned short *__restrict__ in, const float *__restrict__ E,
                                  double *__restrict__ out, long long off, long long n, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long g = off + i;
    const float J = E[g % N] * kInv4PiF;
    out[i] = (double)fmaf(J, __bfloat162float(__ushort_as_bfloat16(in[g])), J);
  }
}

// E = 4 pi sum W I, F = 4 pi sum W n I, P = 4 pi sum W n n I, accumulated
// in double whatever the storage type.
template <typename Real>
__global__ void moments_kernel(const Real *__restrict__ I, const Real *__restrict__ ang, int M, long long N,
                               Real *__restrict__ mom) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = 0; m < M; ++m) {
      double nx = ang[4 * m], ny = ang[4 * m + 1], nz = ang[4 * m + 2];
      double wi = (double)ang[4 * m + 3] * (double)I[(long long)m * N + c];
      s[0] += wi;
      s[1] += nx * wi; s[2] += ny * wi; s[3] += nz * wi;
      s[4] += nx * nx * wi; s[5] += ny * ny * wi; s[6] += nz * nz * wi;
      s[7] += nx * ny * wi; s[8] += nx * nz * wi; s[9] += ny * nz * wi;
    }
    for (int q = 0; q < 10; ++q) mom[(long long)q * N + c] = (Real)(4.0 * kPi * s[q]);
  }
}

__global__ void check_kernel(const double *__restrict__ x, long long n, double lo, int strict, int nzbit, int *flag) {
  int bits = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = x[i];
    if (!isfinite(v) || (strict ? !(v > lo) : !(v >= lo))) bits |= 1;
    if (v != 0.0) bits |= nzbit;
  }
  if (bits) atomicOr(flag, bits);
}

}  // namespace

template <typename Real>
cudaError_t launch_convert_in(const double *src, Real *dst, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  convert_in_kernel<Real><<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_convert_out(const Real *src, double *dst, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  convert_out_kernel<Real><<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_isotropic(const double *T, Real *I, int M, long long N, cudaStream_t s) {
  isotropic_kernel<Real><<<grid_for(N, 256), 256, 0, s>>>(T, I, M, N);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_moments(const Real *I, const Real *ang, int M, long long N, Real *mom, cudaStream_t s) {
  moments_kernel<Real><<<grid_for(N, 256), 256, 0, s>>>(I, ang, M, N, mom);
  return cudaGetLastError();
}

cudaError_t launch_check(const double *x, long long n, double lo, int strict, int nzbit, int *flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, n, lo, strict, nzbit, flag);
  return cudaGetLastError();
}

cudaError_t launch_encode_b16(const float *I, const float *E, unsigned short *out, int M, long long N, cudaStream_t s) {
  encode_b16_kernel<<<grid_for(N, 256), 256, 0, s>>>(I, E, out, M, N);
  return cudaGetLastError();
}

cudaError_t launch_decode_b16(const unsigned short *in, const float *E, double *out, long long off, long long n,
                              long long N, cudaStream_t s) {
  decode_b16_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, E, out, off, n, N);
  return cudaGetLastError();
}

template cudaError_t launch_convert_in<float>(const double *, float *, long long, cudaStream_t);
template cudaError_t launch_convert_in<double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_convert_out<float>(const float *, double *, long long, cudaStream_t);
template cudaError_t launch_convert_out<double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_isotropic<float>(const double *, float *, int, long long, cudaStream_t);
template cudaError_t launch_isotropic<double>(const double *, double *, int, long long, cudaStream_t);
template cudaError_t launch_moments<float>(const float *, const float *, int, long long, float *, cudaStream_t);
template cudaError_t launch_moments<double>(const double *, const double *, int, long long, double *, cudaStream_t);

}  // namespace rtg
