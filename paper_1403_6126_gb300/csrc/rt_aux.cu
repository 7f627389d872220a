// Elementwise device helpers of the runtime: precision conversion, the
// isotropic equilibrium intensity, the sec. 3 quadrature of a given field,
// and input scans.  All grid-stride, sized as a multiple of the SM count.
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

template cudaError_t launch_convert_in<float>(const double *, float *, long long, cudaStream_t);
template cudaError_t launch_convert_in<double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_convert_out<float>(const float *, double *, long long, cudaStream_t);
template cudaError_t launch_convert_out<double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_isotropic<float>(const double *, float *, int, long long, cudaStream_t);
template cudaError_t launch_isotropic<double>(const double *, double *, int, long long, cudaStream_t);
template cudaError_t launch_moments<float>(const float *, const float *, int, long long, float *, cudaStream_t);
template cudaError_t launch_moments<double>(const double *, const double *, int, long long, double *, cudaStream_t);

}  // namespace rtg
