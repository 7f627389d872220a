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

// The same in the quad-interleaved float layout: one float4 per cell and
// quad, angles past M zero.
__global__ void isotropic_quad_kernel(const double *__restrict__ T, float4 *__restrict__ I, int M, long long N) {
  const int NQ = (M + 3) / 4;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const double t = T[c];
    const float b = (float)(t * t * t * t / (4.0 * kPi));
    for (int q = 0; q < NQ; ++q) {
      const int m = 4 * q;
      I[(long long)q * N + c] = make_float4(b, m + 1 < M ? b : 0.0f, m + 2 < M ? b : 0.0f, m + 3 < M ? b : 0.0f);
    }
  }
}

// Angle-major doubles, elements [off, off + n) (element i: angle i / N of
// cell i % N), into the quad layout (element (m, c) at float (m/4) 4N + 4c
// + m%4), and back.
__global__ void quad_in_kernel(const double *__restrict__ src, float *__restrict__ dst, long long off, long long n,
                               long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long g = off + i, m = g / N, c = g - m * N;
    dst[(m >> 2) * 4 * N + 4 * c + (m & 3)] = (float)src[i];
  }
}

__global__ void quad_out_kernel(const float *__restrict__ src, double *__restrict__ dst, long long off, long long n,
                                long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long g = off + i, m = g / N, c = g - m * N;
    dst[i] = (double)src[(m >> 2) * 4 * N + 4 * c + (m & 3)];
  }
}

// bf16 storage: delta = I / J - 1 with J = E / (4 pi) of the cell (the same
// arithmetic as the step kernel's b16_* helpers in rt_step_pair.cuh).
constexpr float kInv4PiF = float(1.0 / (4.0 * 3.14159265358979323846));

__global__ void encode_b16_kernel(const float *__restrict__ I, const double *__restrict__ E,
                                  unsigned short *__restrict__ out, int M, long long N) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const float J = (float)E[c] * kInv4PiF;
    const float rJ = J > 1e-30f ? 1.0f / J : 0.0f;
    for (int m = 0; m < M; ++m) {
      const long long i = (long long)m * N + c;
      out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(fmaf(I[i], rJ, -1.0f)));
    }
  }
}

__global__ void decode_b16_kernel(const unsigned short *__restrict__ in, const double *__restrict__ E,
                                  double *__restrict__ out, long long off, long long n, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long g = off + i;
    const float J = (float)E[g % N] * kInv4PiF;
    out[i] = (double)fmaf(J, __bfloat162float(__ushort_as_bfloat16(in[g])), J);
  }
}

// E = 4 pi sum W I, F = 4 pi sum W n I, P = 4 pi sum W n n I, accumulated
// in double whatever the storage type.
template <typename Real>
__global__ void moments_kernel(const Real *__restrict__ I, const Real *__restrict__ ang, int M, long long N,
                               double *__restrict__ mom) {
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
    for (int q = 0; q < 10; ++q) mom[(long long)q * N + c] = 4.0 * kPi * s[q];
  }
}

// Float intensities (angle-major, or the quad layout when QUAD): products
// in float and each of the ten sums compensated (Kahan), read out as the
// double hi - lo times wscale (1 / sum W for the quad layout's kernels,
// whose sums are over the normalised weights; 1 otherwise).  In double this kernel would run at the FP64 rate (~20 FP64
// operations per cell-angle: milliseconds for a 128^3 x 80 field).
template <bool QUAD>
__global__ void moments_kernel_f(const float *__restrict__ I, const float *__restrict__ ang, int M, long long N,
                                 double wscale, double *__restrict__ mom) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    float hi[10], lo[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) hi[q] = lo[q] = 0.0f;
    for (int m = 0; m < M; ++m) {
      const float nx = ang[4 * m], ny = ang[4 * m + 1], nz = ang[4 * m + 2];
      const float Im = QUAD ? I[(long long)(m >> 2) * 4 * N + 4 * c + (m & 3)] : I[(long long)m * N + c];
      const float wi = ang[4 * m + 3] * Im;
      const float wx = nx * wi, wy = ny * wi, wz = nz * wi;
      const float term[10] = {wi, wx, wy, wz, nx * wx, ny * wy, nz * wz, ny * wx, nz * wx, nz * wy};
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        const float y = term[q] - lo[q];
        const float s = hi[q] + y;
        lo[q] = (s - hi[q]) - y;
        hi[q] = s;
      }
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) mom[(long long)q * N + c] = 4.0 * kPi * wscale * ((double)hi[q] - (double)lo[q]);
  }
}

// The smallest intensity of each cell over its M angles (quad layout,
// padding angles excluded): the center the float step's deviations are
// taken from.
__global__ void centers_kernel(const float4 *__restrict__ I, int M, long long N, float *__restrict__ cen) {
  const int NQ = (M + 3) / 4;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    float mn = I[c].x;
    for (int j = 0; j < NQ; ++j) {
      const float4 q = I[(long long)j * N + c];
      const int left = M - 4 * j;
      mn = fminf(mn, q.x);
      if (left > 1) mn = fminf(mn, q.y);
      if (left > 2) mn = fminf(mn, q.z);
      if (left > 3) mn = fminf(mn, q.w);
    }
    cen[c] = mn;
  }
}

// f = P / E of each cell (sec. 2: f = K/J), one double reciprocal per cell.
__global__ void eddington_kernel(const double *__restrict__ mom, double *__restrict__ f, long long N) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const double E = mom[c];
    const double rE = E != 0.0 ? 1.0 / E : 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) f[(long long)q * N + c] = mom[(long long)(4 + q) * N + c] * rE;
  }
}

// Range tests on the IEEE-754 bit pattern u of a double, in integer
// arithmetic (FP64 compares run at GB300's low FP64 rate): the finite
// values are the patterns with |u| below that of +infinity; the positive
// ones are 0 < u below +infinity; the non-negative ones add -0.
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull, kAbsMask = 0x7FFFFFFFFFFFFFFFull,
                             kNegZero = 0x8000000000000000ull;
__device__ __forceinline__ unsigned long long bits_of(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ bool finite_bits(unsigned long long u) { return (u & kAbsMask) < kInfBits; }
__device__ __forceinline__ bool positive_bits(unsigned long long u) { return u - 1ull < kInfBits - 1ull; }
__device__ __forceinline__ bool nonneg_bits(unsigned long long u) { return u < kInfBits || u == kNegZero; }

__global__ void check_kernel(const double *__restrict__ x, long long n, double lo, int strict, int nzbit, int *flag) {
  int bits = 0;
  const bool zero_lo = lo == 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    const unsigned long long u = bits_of(v);
    const bool ok = zero_lo ? (strict ? positive_bits(u) : nonneg_bits(u))
                            : (finite_bits(u) && (strict ? v > lo : v >= lo));
    if (!ok) bits |= 1;
    if ((u & kAbsMask) != 0) bits |= nzbit;
  }
  // one atomic per block: an atomic per thread on the one flag word would
  // serialize (nearly every thread sets the nonzero bit of a velocity field)
  const int bad = __syncthreads_or(bits & 1), nonzero = __syncthreads_or(bits & nzbit);
  if (threadIdx.x == 0 && (bad || nonzero)) atomicOr(flag, (bad ? 1 : 0) | (nonzero ? nzbit : 0));
}

// Gas fields staged as doubles (stage: rho, T, v_x, v_y, v_z, sigma_a,
// sigma_s, N each), cells [c0, c0 + n): bit 0 of *flag for a value out of
// range (rho, T > 0; sigma >= 0; all finite), bit 1 for a nonzero velocity;
// with CONVERT also the context's arrays (Real, T in double).
template <typename Real, bool CONVERT>
__global__ void fields_in_kernel(const double *__restrict__ stage, long long N, long long c0, long long n,
                                 Real *__restrict__ rho, Real *__restrict__ sa, Real *__restrict__ ss,
                                 Real *__restrict__ v, double *__restrict__ T, int *flag) {
  int bits = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long i = c0 + k;
    const double r = stage[i], t = stage[N + i], vx = stage[2 * N + i], vy = stage[3 * N + i],
                 vz = stage[4 * N + i], a = stage[5 * N + i], s = stage[6 * N + i];
    const unsigned long long ux = bits_of(vx), uy = bits_of(vy), uz = bits_of(vz);
    if (!(positive_bits(bits_of(r)) && positive_bits(bits_of(t)) && nonneg_bits(bits_of(a)) &&
          nonneg_bits(bits_of(s)) && finite_bits(ux) && finite_bits(uy) && finite_bits(uz)))
      bits |= 1;
    if (((ux | uy | uz) & kAbsMask) != 0) bits |= 2;
    if (CONVERT) {
      rho[i] = (Real)r;
      sa[i] = (Real)a;
      ss[i] = (Real)s;
      v[i] = (Real)vx;
      v[N + i] = (Real)vy;
      v[2 * N + i] = (Real)vz;
      T[i] = t;
    }
  }
  const int bad = __syncthreads_or(bits & 1), nonzero = __syncthreads_or(bits & 2);
  if (threadIdx.x == 0 && (bad || nonzero)) atomicOr(flag, (bad ? 1 : 0) | (nonzero ? 2 : 0));
}


}  // namespace

template <typename Real>
cudaError_t launch_fields_in(const double *stage, long long N, long long c0, long long n, bool convert, Real *rho,
                             Real *sa, Real *ss, Real *v, double *T, int *flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (convert)
    fields_in_kernel<Real, true><<<grid_for(n, 256), 256, 0, s>>>(stage, N, c0, n, rho, sa, ss, v, T, flag);
  else
    fields_in_kernel<Real, false><<<grid_for(n, 256), 256, 0, s>>>(stage, N, c0, n, rho, sa, ss, v, T, flag);
  return cudaGetLastError();
}


template cudaError_t launch_fields_in<float>(const double *, long long, long long, long long, bool, float *, float *,
                                             float *, float *, double *, int *, cudaStream_t);
template cudaError_t launch_fields_in<double>(const double *, long long, long long, long long, bool, double *,
                                              double *, double *, double *, double *, int *, cudaStream_t);

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
cudaError_t launch_isotropic(const double *T, Real *I, int M, long long N, bool quad, cudaStream_t s) {
  if constexpr (sizeof(Real) == 4) {
    if (quad) {
      isotropic_quad_kernel<<<grid_for(N, 256), 256, 0, s>>>(T, reinterpret_cast<float4 *>(I), M, N);
      return cudaGetLastError();
    }
  }
  isotropic_kernel<Real><<<grid_for(N, 256), 256, 0, s>>>(T, I, M, N);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_moments(const Real *I, const Real *ang, int M, long long N, bool quad, double wscale, double *mom,
                           cudaStream_t s) {
  if constexpr (sizeof(Real) == 4) {
    if (quad)
      moments_kernel_f<true><<<grid_for(N, 256), 256, 0, s>>>(I, ang, M, N, wscale, mom);
    else
      moments_kernel_f<false><<<grid_for(N, 256), 256, 0, s>>>(I, ang, M, N, wscale, mom);
  } else {
    moments_kernel<Real><<<grid_for(N, 256), 256, 0, s>>>(I, ang, M, N, mom);
  }
  return cudaGetLastError();
}

cudaError_t launch_centers(const float *I, int M, long long N, float *cen, cudaStream_t s) {
  centers_kernel<<<grid_for(N, 256), 256, 0, s>>>(reinterpret_cast<const float4 *>(I), M, N, cen);
  return cudaGetLastError();
}

cudaError_t launch_eddington(const double *mom, double *f, long long N, cudaStream_t s) {
  eddington_kernel<<<grid_for(N, 256), 256, 0, s>>>(mom, f, N);
  return cudaGetLastError();
}

cudaError_t launch_quad_in(const double *src, float *dst, long long off, long long n, long long N, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  quad_in_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst, off, n, N);
  return cudaGetLastError();
}

cudaError_t launch_quad_out(const float *src, double *dst, long long off, long long n, long long N, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  quad_out_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst, off, n, N);
  return cudaGetLastError();
}

cudaError_t launch_check(const double *x, long long n, double lo, int strict, int nzbit, int *flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, n, lo, strict, nzbit, flag);
  return cudaGetLastError();
}

cudaError_t launch_encode_b16(const float *I, const double *E, unsigned short *out, int M, long long N, cudaStream_t s) {
  encode_b16_kernel<<<grid_for(N, 256), 256, 0, s>>>(I, E, out, M, N);
  return cudaGetLastError();
}

cudaError_t launch_decode_b16(const unsigned short *in, const double *E, double *out, long long off, long long n,
                              long long N, cudaStream_t s) {
  decode_b16_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, E, out, off, n, N);
  return cudaGetLastError();
}

template cudaError_t launch_convert_in<float>(const double *, float *, long long, cudaStream_t);
template cudaError_t launch_convert_in<double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_convert_out<float>(const float *, double *, long long, cudaStream_t);
template cudaError_t launch_convert_out<double>(const double *, double *, long long, cudaStream_t);
template cudaError_t launch_isotropic<float>(const double *, float *, int, long long, bool, cudaStream_t);
template cudaError_t launch_isotropic<double>(const double *, double *, int, long long, bool, cudaStream_t);
template cudaError_t launch_moments<float>(const float *, const float *, int, long long, bool, double, double *,
                                           cudaStream_t);
template cudaError_t launch_moments<double>(const double *, const double *, int, long long, bool, double, double *,
                                            cudaStream_t);

}  // namespace rtg
