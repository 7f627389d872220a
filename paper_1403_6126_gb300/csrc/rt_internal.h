// Internal declarations shared by the host runtime and the device kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rtg {

constexpr int kMaxAngles = 256;
constexpr int kMomComps = 10;  // E, Fx, Fy, Fz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz

// Everything one fused step launch needs.  Real is the intensity and
// transport type (double for the FP64 path, float for the mixed path);
// temperature and the gas energy source are always double.
template <typename Real>
struct StepArgs {
  int dim;            // active axes
  int n[3];           // cells per axis (1 on inactive axes)
  int M;              // angles
  long long N;        // cells
  int bc[3][2];       // boundary kinds per axis / side
  Real C, invC, P;    // Crat, 1/Crat, Prat
  Real dt;            // time step
  Real dtdx[3];       // dt / dx_d
  Real dx[3];         // cell sizes
  double dt_d, kv_per_rho;  // dt and R/(gamma-1) in double
  int hold_T, estimate_v;
  int newton_max_it;  // Newton on T: iteration cap and stopping tolerance
  double newton_rtol;
  Real wnorm;         // 1 - 1 / (sum of the weights as the float table holds them)
  float msum[10][2];  // the float table's normalised quadrature sums (table_moment_sums)
  const Real *ang;    // [M][4]: n_x, n_y, n_z, W
  const Real *inflow; // [3][2][M]
  // Intensities.  Double: angle-major [M][N].  Float: quad-interleaved,
  // ceil(M/4) planes of float4 ([q][c] holds angles 4q .. 4q+3 of cell c,
  // angles past M zero).
  const Real *I_in;
  Real *I_out;
  const Real *rho, *sa, *ss;  // [N]
  const Real *v;      // [3][N]
  const double *T_in; // [N]
  double *T_out;      // [N]
  const double *mom_in;  // [10][N] moments of I_in
  double *mom_out;       // [10][N] moments of I_out
  // Float quad layout: each cell's smallest intensity over its angles, of
  // I_in (read) and of I_out (written); null: formed from I_in in the kernel
  // and not written.
  const float *cen_in;
  float *cen_out;
  double *dEgas;      // [N]
  double *dMom;       // [3][N]
  int *status;        // [0]: cells whose T Newton failed
  // bf16 storage (RT_BF16, float kernels only): the stored value of angle m
  // in cell c (angle-major [M][N]) is delta = I / J - 1 with J = E / (4 pi)
  // of the cell's stored moments; I_in / I_out are unused then and Q is a
  // float [M][N] scratch for the right-hand sides Q_m.  Null otherwise.
  const unsigned short *I16_in;
  unsigned short *I16_out;
  float *Q;
  // The launch covers tile layers [outer_begin, outer_begin + outer_count)
  // along the outermost active axis (z in 3-D, y in 2-D, x in 1-D;
  // outer_count = 0: every layer).  Tiles are independent within a step, so
  // a grid stepped in slabs gives bitwise the whole-grid result.
  int outer_begin, outer_count;
};

// The float kernels take their angle sums over the weights of the float
// table ang4 ([M][4], W in slot 3) divided by their sum S (1 + O(1e-8) after
// rounding each weight), so that the weights they use sum to exactly 1.
// weight_norm returns 1 - 1/S, S summed in double (exact for comparable
// weights) and the result rounded to float once.
inline double weight_sum(const float *ang4, int M) {
  double s = 0.0;
  for (int m = 0; m < M; ++m) s += (double)ang4[4 * m + 3];
  return s;
}
inline float weight_norm(const float *ang4, int M) { return (float)(1.0 - 1.0 / weight_sum(ang4, M)); }

// The quadrature sums of a float angle table ang4 ([M][4]: n_x, n_y, n_z,
// W) that the float kernels' moments are taken against, over the normalised
// weights W / S (see weight_norm): sum W (1), sum W n_i (x, y, z), sum W n_i
// n_j (xx, yy, zz, xy, xz, yz), each summed in double and split into a float
// pair (hi, lo).
inline void table_moment_sums(const float *ang4, int M, float out[10][2]) {
  double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int m = 0; m < M; ++m) {
    const double x = ang4[4 * m], y = ang4[4 * m + 1], z = ang4[4 * m + 2], W = ang4[4 * m + 3];
    s[0] += W;
    s[1] += W * x; s[2] += W * y; s[3] += W * z;
    s[4] += W * x * x; s[5] += W * y * y; s[6] += W * z * z;
    s[7] += W * x * y; s[8] += W * x * z; s[9] += W * y * z;
  }
  for (int k = 0; k < 10; ++k) {
    const double v = s[k] / s[0];
    out[k][0] = (float)v;
    out[k][1] = (float)(v - (double)out[k][0]);
  }
}

struct TileShape {
  int tx, ty, tz;
};

// Launch the fused step; returns the CUDA error of the launch.
template <typename Real>
cudaError_t launch_step(const StepArgs<Real> &a, int dim, bool has_v, TileShape tile, cudaStream_t s);

// Pick a tile shape that fits shared memory for (dim, M, has_v); false if
// even the smallest tile does not fit.
template <typename Real>
bool choose_tile(int dim, int M, bool has_v, TileShape *out);

// Whether a tile shape can be launched: thread count within the kernel's
// launch bound, shared memory within the opt-in limit, and enough staging
// slots for its halo.
template <typename Real>
bool tile_ok(int dim, int M, bool has_v, TileShape t);

// The compiled shapes that can run (dim, M, has_v), preferred first; out
// holds up to 8.  Returns their count.
template <typename Real>
int tile_candidates(int dim, int M, bool has_v, TileShape *out);

// The bf16-storage step (RT_BF16): one compiled tile per dimension (16x8x4,
// 32x16, 512); choose_tile_b16 gives it, or false when its shared memory
// does not fit M angles.
cudaError_t launch_b16(const StepArgs<float> &a, int dim, bool vel, TileShape t, cudaStream_t s);
bool choose_tile_b16(int dim, int M, TileShape *out);

// The float step on the quad-interleaved layout (RT_FP32).  host_ang [M][4]
// and host_inflow [6][M] are the float tables the device holds: for M <= 80
// they travel as a launch-parameter table, larger sets read the device
// tables a.ang / a.inflow into shared memory.
cudaError_t launch_step_quad(const StepArgs<float> &a, const float *host_ang, const float *host_inflow, int dim,
                             bool vel, TileShape t, cudaStream_t s);

// Elementwise helpers (all stream-ordered).
template <typename Real>
cudaError_t launch_convert_in(const double *src, Real *dst, long long n, cudaStream_t s);
template <typename Real>
cudaError_t launch_convert_out(const Real *src, double *dst, long long n, cudaStream_t s);
// Isotropic equilibrium T^4/(4 pi): angle-major [M][N] (double), or the
// quad-interleaved float layout with zero padding (quad = true).
template <typename Real>
cudaError_t launch_isotropic(const double *T, Real *I, int M, long long N, bool quad, cudaStream_t s);
// E, F, P (double [10][N]) of an intensity field (angle-major, or the quad
// layout when quad is set), times wscale (float intensities only).
template <typename Real>
cudaError_t launch_moments(const Real *I, const Real *ang, int M, long long N, bool quad, double wscale, double *mom,
                           cudaStream_t s);
// Each cell's smallest intensity over its M angles (quad layout) into cen [N].
cudaError_t launch_centers(const float *I, int M, long long N, float *cen, cudaStream_t s);
// Eddington tensor f = P / E (6 components, [6][N]) from stored moments
// [10][N]; 0 where E = 0.
cudaError_t launch_eddington(const double *mom, double *f, long long N, cudaStream_t s);
// Elements [off, off + n) of an angle-major double field (element i is angle
// i / N of cell i % N) into / out of the quad-interleaved float layout.
cudaError_t launch_quad_in(const double *src, float *dst, long long off, long long n, long long N, cudaStream_t s);
cudaError_t launch_quad_out(const float *src, double *dst, long long off, long long n, long long N, cudaStream_t s);

// bf16 storage: encode a float intensity array [M][N] as deviations from
// the mean intensity of each cell (E [N] its energy density), and decode
// elements [off, off + n) of a stored array to doubles.
cudaError_t launch_encode_b16(const float *I, const double *E, unsigned short *out, int M, long long N, cudaStream_t s);
cudaError_t launch_decode_b16(const unsigned short *in, const double *E, double *out, long long off, long long n,
                              long long N, cudaStream_t s);

// Scans n doubles: ORs bit 0 into *flag for a non-finite value or one below
// `lo` (or equal to it when strict), and ORs `nzbit` for a nonzero value.
cudaError_t launch_check(const double *x, long long n, double lo, int strict, int nzbit, int *flag, cudaStream_t s);
// Scan of the gas fields staged as doubles (stage: rho, T, v_x, v_y, v_z,
// sigma_a, sigma_s, N each) over cells [c0, c0 + n) into *flag (bit 0: a
// value out of range, bit 1: some v != 0); with convert also the copy into
// the context's arrays (rho, sigma_a, sigma_s, v in Real; T in double).
template <typename Real>
cudaError_t launch_fields_in(const double *stage, long long N, long long c0, long long n, bool convert, Real *rho,
                             Real *sa, Real *ss, Real *v, double *T, int *flag, cudaStream_t s);

}  // namespace rtg
