// Fused radiation-transfer step for sm_103a (Jiang, Stone & Davis 2014,
// arXiv:1403.6126, secs. 3-4).
//
// One CTA owns a tile of cells (one thread per cell) and walks the angles.
// For every angle it stages the tile's intensity plus a two-cell halo on each
// active axis in shared memory (boundary values applied while staging),
// computes the transport change Delta F_m of its cell (sec. 4.2), folds it
// into the right-hand side of the implicit step it belongs to, accumulates
// every angle sum the implicit solves need, and keeps one value per
// cell-angle (Q_m below) in shared memory.  After the last angle each thread
// solves its cell: the T^4 energy equation of Step 4 (sec. 4.3) reduced to a
// scalar quartic, the 2x2 system of Step 5 (sec. 4.4), and then writes
// I^{n+1}, the moments E_r, F_r, P_r (sec. 3) and the gas sources.  I is
// read once and written once per step.
//
// Reduction used (both implicit steps are linear in I for fixed T):
//   Step 4 row m:  d_m I_m = r_m + e_m theta - kappa S,   theta = T^4/(4 pi)
//     d_m = 1 + dt C sa - dt sa vn_m,  e_m = dt sa (C + 3 vn_m),
//     kappa = dt sa / C,  S = sum_l g_l I_l,  g_l = W_l (v.v + vn_l^2),
//     vn_m = n_m . v~ ;
//   Step 5 (unknowns x = W I): a_m x_m + sum_l (b_l + c_m) x_l = r'_m with
//     r'_m = I4_m (+ Delta F_m when sigma_s > sigma_a),
//     I4_m = Q_m + (e_m/d_m) theta - kappa S / d_m,
//     Q_m  = r_m / d_m (+ Delta F_m when sigma_s > sigma_a).
// Every angle sum is linear in Q_m with coefficients that depend only on
// the cell and the angle, so all of them are accumulated in the same pass
// that computes the transport.
#include <math.h>

#include "rt_internal.h"

namespace rtg {

namespace {

constexpr int kHalo = 2;
constexpr double kPi = 3.14159265358979323846;

enum { BC_PERIODIC = 0, BC_VACUUM = 1, BC_COPY = 2, BC_INFLOW = 3 };

// Box-cell source word: low 28 bits = cell index, bits 28..30 = ghost code
// (0 interior, 1 + 2*axis + side for a cell outside along one axis);
// -1 = box corner cell that the cross-shaped stencil never reads.
constexpr int kIdxBits = 28;
constexpr int kIdxMask = (1 << kIdxBits) - 1;

__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

__device__ __forceinline__ float alpha_of(float dl, float st) {
  float s = 10.0f * dl * st;
  float tau = s * s;
  if (tau < 1e-12f) return 1.0f;
  return sqrtf(-expm1f(-tau) / tau);
}
__device__ __forceinline__ double alpha_of(double dl, double st) {
  double s = 10.0 * dl * st;
  double tau = s * s;
  if (tau < 1e-12) return 1.0;
  return sqrt(-expm1(-tau) / tau);
}

// van Leer slope: harmonic mean of one-sided differences of equal sign.
template <typename R>
__device__ __forceinline__ R vl_slope(R qm, R q0, R qp) {
  R dl = q0 - qm, dr = qp - q0;
  R pr = dl * dr;
  return pr > R(0) ? R(2) * pr * fast_rcp(dl + dr) : R(0);
}

// Compensated accumulator: terms go into a plain partial sum which is
// folded into (hi, lo) by Kahan's rule every few angles.
template <typename R>
struct KSum {
  R part, hi, lo;
  __device__ __forceinline__ void zero() { part = hi = lo = R(0); }
  __device__ __forceinline__ void fold() {
    R y = part - lo;
    R t = hi + y;
    lo = (t - hi) - y;
    hi = t;
    part = R(0);
  }
  __device__ __forceinline__ R total() {
    fold();
    return hi;
  }
};
// Double precision needs no compensation; it sums in angle order like the
// oracle does.
template <>
struct KSum<double> {
  double part;
  __device__ __forceinline__ void zero() { part = 0.0; }
  __device__ __forceinline__ void fold() {}
  __device__ __forceinline__ double total() { return part; }
};

__device__ __forceinline__ int map_coord(int g, int n, int kind_lo, int kind_hi) {
  if (g < 0) return kind_lo == BC_PERIODIC ? ((g % n) + n) % n : 0;
  if (g >= n) return kind_hi == BC_PERIODIC ? g % n : n - 1;
  return g;
}

template <typename Real, int DIM>
struct Layout {
  int TX, TY, TZ, BX, BY, BZ, nbox, ncell, nf[3];
  __device__ __forceinline__ void init() {
    TX = blockDim.x; TY = blockDim.y; TZ = blockDim.z;
    BX = TX + 2 * kHalo;
    BY = DIM >= 2 ? TY + 2 * kHalo : 1;
    BZ = DIM >= 3 ? TZ + 2 * kHalo : 1;
    nbox = BX * BY * BZ;
    ncell = TX * TY * TZ;
    nf[0] = (TX + 1) * TY * TZ;
    nf[1] = DIM >= 2 ? TX * (TY + 1) * TZ : 0;
    nf[2] = DIM >= 3 ? TX * TY * (TZ + 1) : 0;
  }
};

// Shared-memory bytes of one CTA (host and device agree on this).
__host__ __device__ inline size_t smem_bytes(int dim, int M, bool has_v, int tx, int ty, int tz, size_t rs) {
  size_t BX = tx + 2 * kHalo, BY = dim >= 2 ? ty + 2 * kHalo : 1, BZ = dim >= 3 ? tz + 2 * kHalo : 1;
  size_t nbox = BX * BY * BZ, ncell = (size_t)tx * ty * tz;
  size_t nf = (size_t)(tx + 1) * ty * tz + (dim >= 2 ? (size_t)tx * (ty + 1) * tz : 0) +
              (dim >= 3 ? (size_t)tx * ty * (tz + 1) : 0);
  size_t reals = 4 * (size_t)M + (size_t)M * ncell + nbox * (has_v ? 5 : 1) + nf * (has_v ? 2 : 1);
  return reals * rs + nbox * sizeof(int) + 16;
}

template <typename Real, int DIM, bool VEL>
__global__ void __launch_bounds__(512) step_kernel(const StepArgs<Real> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Layout<Real, DIM> L;
  L.init();
  const int M = a.M;
  const long long N = a.N;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tid = threadIdx.x + L.TX * (threadIdx.y + L.TY * threadIdx.z);
  const int nthr = L.ncell;

  Real *s_ang = reinterpret_cast<Real *>(smem_raw);
  Real *s_Q = s_ang + 4 * M;
  Real *s_It = s_Q + (size_t)M * L.ncell;
  Real *s_IV = s_It + L.nbox;                      // VEL only
  Real *s_w = s_IV + (VEL ? L.nbox : 0);           // VEL only: 3 * nbox
  Real *s_af = s_w + (VEL ? 3 * L.nbox : 0);       // face alpha, all axes
  const int nft = L.nf[0] + L.nf[1] + L.nf[2];
  Real *s_vf = s_af + nft;                         // VEL only: face velocity
  int *s_src = reinterpret_cast<int *>(s_vf + (VEL ? nft : 0));

  const int x0 = blockIdx.x * L.TX, y0 = blockIdx.y * L.TY, z0 = blockIdx.z * L.TZ;

  // ---- per-tile setup: angle table, box source words, face data ----------
  for (int i = tid; i < 4 * M; i += nthr) s_ang[i] = a.ang[i];
  for (int b = tid; b < L.nbox; b += nthr) {
    int bx = b % L.BX, by = (b / L.BX) % L.BY, bz = b / (L.BX * L.BY);
    int g[3] = {x0 - kHalo + bx, DIM >= 2 ? y0 - kHalo + by : 0, DIM >= 3 ? z0 - kHalo + bz : 0};
    int nout = 0, code = 0;
    for (int d = 0; d < DIM; ++d) {
      if (g[d] < 0 || g[d] >= a.n[d]) {
        ++nout;
        code = 1 + 2 * d + (g[d] >= a.n[d] ? 1 : 0);
        g[d] = map_coord(g[d], a.n[d], a.bc[d][0], a.bc[d][1]);
      }
    }
    long long c = g[0] + (long long)nx * (g[1] + (long long)ny * g[2]);
    s_src[b] = nout > 1 ? -1 : (int)(c | ((long long)code << kIdxBits));
    if (VEL) {
      // w = 3 J v with J = E / (4 pi): the IV of angle m is n_m . w
      Real w3 = 0, vx = 0, vy = 0, vz = 0;
      if (nout <= 1) {
        w3 = Real(3.0 / (4.0 * kPi)) * a.mom_in[c];
        vx = a.v[c]; vy = a.v[N + c]; vz = a.v[2 * N + c];
      }
      s_w[b] = w3 * vx; s_w[L.nbox + b] = w3 * vy; s_w[2 * L.nbox + b] = w3 * vz;
    }
  }
  {
    // faces of axis d: face l (between local cells l-1 and l along d)
    int off = 0;
    for (int d = 0; d < DIM; ++d) {
      const int Td = d == 0 ? L.TX : (d == 1 ? L.TY : L.TZ);
      const int To1 = d == 0 ? L.TY : L.TX;
      for (int f = tid; f < L.nf[d]; f += nthr) {
        int l = f % (Td + 1), rest = f / (Td + 1);
        int o1 = rest % To1, o2 = rest / To1;
        int loc[3];
        loc[d] = l;
        if (d == 0) { loc[1] = o1; loc[2] = o2; }
        else if (d == 1) { loc[0] = o1; loc[2] = o2; }
        else { loc[0] = o1; loc[1] = o2; }
        int g[3] = {x0 + loc[0], DIM >= 2 ? y0 + loc[1] : 0, DIM >= 3 ? z0 + loc[2] : 0};
        Real al[2], vd[2];
        for (int side = 0; side < 2; ++side) {
          int gg[3] = {g[0], g[1], g[2]};
          gg[d] = g[d] - 1 + side;
          // clamp the other axes into the grid (ragged tiles; unused faces)
          for (int e = 0; e < DIM; ++e)
            if (e != d) gg[e] = min(gg[e], a.n[e] - 1);
          gg[d] = map_coord(gg[d], a.n[d], a.bc[d][0], a.bc[d][1]);
          long long c = gg[0] + (long long)nx * (gg[1] + (long long)ny * gg[2]);
          al[side] = alpha_of(a.dx[d], a.sa[c] + a.ss[c]);
          vd[side] = VEL ? a.v[d * N + c] : Real(0);
        }
        s_af[off + f] = Real(0.5) * (al[0] + al[1]);
        if (VEL) s_vf[off + f] = Real(0.5) * (vd[0] + vd[1]);
      }
      off += L.nf[d];
    }
  }

  // ---- own cell --------------------------------------------------------------
  const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
  const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
  const bool valid = gx < nx && (DIM < 2 || gy < ny) && (DIM < 3 || gz < nz);
  const long long c = valid ? gx + (long long)nx * (gy + (long long)ny * gz) : 0;
  const int bo = (lx + kHalo) + L.BX * ((DIM >= 2 ? ly + kHalo : 0) + L.BY * (DIM >= 3 ? lz + kHalo : 0));
  const int bstride[3] = {1, L.BX, L.BX * L.BY};
  int fidx_lo[3], fstride[3];
  {
    int off = 0;
    fidx_lo[0] = lx + (L.TX + 1) * (ly + L.TY * lz);
    fstride[0] = 1;
    off += L.nf[0];
    if (DIM >= 2) {
      fidx_lo[1] = off + ly + (L.TY + 1) * (lx + L.TX * lz);
      fstride[1] = 1;
      off += L.nf[1];
    }
    if (DIM >= 3) {
      fidx_lo[2] = off + lz + (L.TZ + 1) * (lx + L.TX * ly);
      fstride[2] = 1;
    }
  }

  const Real C = a.C, invC = a.invC, dt = a.dt;
  Real rho = 1, sa = 0, ss = 0, vt[3] = {0, 0, 0}, vin[3] = {0, 0, 0};
  double T0 = 1.0;
  if (valid) {
    rho = a.rho[c]; sa = a.sa[c]; ss = a.ss[c];
    T0 = a.T_in[c];
    if (VEL) {
      for (int d = 0; d < 3; ++d) vin[d] = a.v[d * N + c];
      if (a.estimate_v) {
        // Step 3 (sec. 4.5): per axis, the backward-Euler momentum exchange
        // with E, F, P_dd held at their step-n values.
        const Real E = a.mom_in[c];
        const Real h = Real(0.5) * dt * (sa + ss);
        for (int d = 0; d < 3; ++d) {
          const Real Fd = a.mom_in[(1 + d) * N + c], Pdd = a.mom_in[(4 + d) * N + c];
          Real num = rho * vin[d] + h * (C * rho * vin[d] + a.P * Fd);
          Real den = rho + h * (C * rho + a.P * (E + Pdd) / C);
          vt[d] = num / den;
        }
      } else {
        vt[0] = vin[0]; vt[1] = vin[1]; vt[2] = vin[2];
      }
    }
  }
  const bool to_scat = ss > sa;
  const Real v2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
  // Step 4 coefficients
  const Real A0 = Real(1) + dt * C * sa, A1 = dt * sa, kap = dt * sa / C;
  // Step 5 coefficients: a'_m = a0 - a1 vn (a_m = a'_m / W_m),
  // b_m = bq0 + vn (bq1 + bq2 vn), c_m = cq vn
  const Real a0 = Real(1) + dt * C * ss, a1 = dt * ss;
  const Real bq0 = -dt * C * ss - dt * ss * v2 / C, bq1 = Real(2) * dt * ss, bq2 = -dt * ss / C;
  const Real cq = Real(-3) * dt * ss;

  // Step 4 sums (sec. 4.3) and Step 5 sums (sec. 4.4); names: <weight><what>
  KSum<Real> sWr, sVr, sGr, sAQ, sBQ;          // depend on the intensities
  Real We = 0, W1 = 0, Ve = 0, V1 = 0, Ge = 0, G1 = 0, Wq = 0;   // cell + angle only
  Real Ap = 0, Ad = 0, Bp = 0, Bd = 0, As1 = 0, Acc = 0, B1p = 0, Bcc = 0;
  KSum<Real> pre[3];                            // sum W n (I^n + Delta F)
  sWr.zero(); sVr.zero(); sGr.zero(); sAQ.zero(); sBQ.zero();
  for (int d = 0; d < 3; ++d) pre[d].zero();

  __syncthreads();

  for (int m = 0; m < M; ++m) {
    const Real nxm = s_ang[4 * m], nym = s_ang[4 * m + 1], nzm = s_ang[4 * m + 2], Wm = s_ang[4 * m + 3];
    // ---- stage I_m (with boundary values) for the tile + halo -----------
    for (int b = tid; b < L.nbox; b += nthr) {
      const int src = s_src[b];
      Real It = 0, IV = 0;
      if (src >= 0) {
        const long long cc = src & kIdxMask;
        const int code = src >> kIdxBits;
        Real I = a.I_in[(long long)m * N + cc];
        if (code) {
          const int axis = (code - 1) >> 1, side = (code - 1) & 1;
          const int kind = a.bc[axis][side];
          if (kind == BC_VACUUM || kind == BC_INFLOW) {
            const Real mu = s_ang[4 * m + axis];
            const bool incoming = side ? (mu < Real(0)) : (mu > Real(0));
            if (incoming) I = kind == BC_VACUUM ? Real(0) : a.inflow[(axis * 2 + side) * M + m];
          }
        }
        if (VEL) {
          IV = nxm * s_w[b] + nym * s_w[L.nbox + b] + nzm * s_w[2 * L.nbox + b];
          It = I - IV * invC;
        } else {
          It = I;
        }
      }
      s_It[b] = It;
      if (VEL) s_IV[b] = IV;
    }
    __syncthreads();

    if (valid) {
      // ---- Step 2 (sec. 4.2): Delta F_m of this cell ----------------------
      Real dF = 0;
      const Real nm[3] = {nxm, nym, nzm};
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const int s = bstride[d];
        const Real mu = nm[d];
        const Real q0 = s_It[bo - 2 * s], q1 = s_It[bo - s], q2 = s_It[bo], q3 = s_It[bo + s], q4 = s_It[bo + 2 * s];
        const Real sl0 = vl_slope(q0, q1, q2), sl1 = vl_slope(q1, q2, q3), sl2 = vl_slope(q2, q3, q4);
        const Real cmu = C * (mu < Real(0) ? -mu : mu) * a.dtdx[d];
        Real flux[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {  // k = 0: face i-1/2, k = 1: face i+1/2
          const Real af = s_af[fidx_lo[d] + k * fstride[d]];
          const Real nu = af * cmu;
          const Real hl = Real(0.5) * (Real(1) - nu);
          const Real left = (k ? q2 : q1) + hl * (k ? sl1 : sl0);
          const Real right = (k ? q3 : q2) - hl * (k ? sl2 : sl1);
          const Real up = mu > Real(0) ? left : right, down = mu > Real(0) ? right : left;
          flux[k] = C * mu * (Real(0.5) * (Real(1) + af) * up + Real(0.5) * (Real(1) - af) * down);
        }
        if (VEL) {
          const Real p0 = s_IV[bo - 2 * s], p1 = s_IV[bo - s], p2 = s_IV[bo], p3 = s_IV[bo + s], p4 = s_IV[bo + 2 * s];
          const Real t0 = vl_slope(p0, p1, p2), t1 = vl_slope(p1, p2, p3), t2 = vl_slope(p2, p3, p4);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const Real vf = s_vf[fidx_lo[d] + k * fstride[d]];
            const Real nv = (vf < Real(0) ? -vf : vf) * a.dtdx[d];
            const Real hl = Real(0.5) * (Real(1) - nv);
            const Real lv = (k ? p2 : p1) + hl * (k ? t1 : t0);
            const Real rv = (k ? p3 : p2) - hl * (k ? t2 : t1);
            const Real ivf = vf > Real(0) ? lv : (vf < Real(0) ? rv : Real(0.5) * (lv + rv));
            flux[k] += mu * ivf;
          }
        }
        dF -= a.dtdx[d] * (flux[1] - flux[0]);
      }

      // ---- fold into the implicit right-hand sides and the sums ------------
      const Real I0 = a.I_in[(long long)m * N + c];
      const Real full = I0 + dF;
      const Real vn = VEL ? nxm * vt[0] + nym * vt[1] + nzm * vt[2] : Real(0);
      const Real dm = A0 - A1 * vn;
      const Real rd = fast_rcp(dm);
      const Real pe = A1 * (C + Real(3) * vn) * rd;          // e_m / d_m
      const Real qa = (to_scat ? I0 : full) * rd;           // r_m / d_m
      const Real Q = to_scat ? qa + dF : qa;
      s_Q[(size_t)m * L.ncell + tid] = Q;
      const Real Wvn = Wm * vn;
      const Real g = Wm * (v2 + vn * vn);
      sWr.part += Wm * qa; We += Wm * pe; W1 += Wm * rd;
      Wq += Wm * (Real(1) - Real(4) * A1 * vn) * rd;
      if (VEL) {
        sVr.part += Wvn * qa; Ve += Wvn * pe; V1 += Wvn * rd;
        sGr.part += g * qa; Ge += g * pe; G1 += g * rd;
      }
      const Real ap = a0 - a1 * vn;
      const Real wa = Wm * fast_rcp(ap);                     // 1 / a_m
      const Real bm = bq0 + vn * (bq1 + bq2 * vn);
      const Real cm = cq * vn;
      const Real bwa = bm * wa;
      sAQ.part += wa * Q; Ap += wa * pe; Ad += wa * rd; As1 += wa; Acc += cm * wa;
      // 1 + sum b/a = sum W (a' + b) / a' (sum W = 1): the dt C sigma_s parts
      // of a' and b cancel analytically instead of in rounding
      const Real apb = Real(1) + a1 * vn - a1 * (v2 + vn * vn) * invC;
      sBQ.part += bwa * Q; Bp += bwa * pe; Bd += bwa * rd; B1p += wa * apb; Bcc += cm * bwa;
      pre[0].part += Wm * nxm * full; pre[1].part += Wm * nym * full; pre[2].part += Wm * nzm * full;
      if ((m & 7) == 7) {
        sWr.fold(); sVr.fold(); sGr.fold(); sAQ.fold(); sBQ.fold();
        pre[0].fold(); pre[1].fold(); pre[2].fold();
      }
    }
    __syncthreads();
  }

  if (!valid) return;

  // ---- Step 4 solve: S, J, v.H affine in theta; scalar quartic in T ---------
  const Real Wr = sWr.total(), Vr = sVr.total(), Gr = sGr.total();
  const Real den = Real(1) + kap * G1;
  const Real S0 = Gr / den, S1 = Ge / den;
  const Real J0 = Wr - kap * S0 * W1;
  const Real H0 = Vr - kap * S0 * V1, H1 = Ve - kap * S1 * V1;
  const Real omJ1 = Wq + kap * S1 * W1;   // 1 - dJ/dtheta, cancellation-free
  const double kv = (double)rho * a.kv_per_rho;
  double T1 = T0;
  if (!a.hold_T) {
    const Real beta = a.P * C * (Real(1) - v2 * invC * invC) * sa;
    const Real c0r = dt * (Real(8.0 * kPi) * a.P * sa * (H0 - S0 * invC) - Real(4.0 * kPi) * beta * J0);
    const Real c4 = dt * (Real(2) * a.P * sa * (H1 - S1 * invC) + beta * omJ1);
    bool ok = false;
    if constexpr (sizeof(Real) == 8) {
      // same iteration and stopping rule as the FP64 reference: Newton from
      // T^n until |dT| <= 1e-13 T, then one more step
      const double c0 = (double)c0r - kv * T0, c4d = (double)c4;
      double T = T0;
      int extra = -1, it;
      for (it = 0; it < 60; ++it) {
        double T3 = T * T * T;
        double f = c4d * T3 * T + kv * T + c0;
        double fp = 4.0 * c4d * T3 + kv;
        double Tn = T - f / fp;
        if (!(Tn > 0)) Tn = 0.5 * T;
        double dT = Tn - T;
        T = Tn;
        if (extra == 0) break;
        if (extra < 0 && fabs(dT) <= 1e-13 * T) extra = 0;
      }
      ok = it < 60;
      T1 = T;
    } else {
      // Newton on delta = T - T^n in float, then one double-precision step
      // (the converged float iterate is within ~1e-7 of the root, so one
      // Newton step in double brings delta to double accuracy)
      const float T0f = (float)T0, kvf = (float)kv;
      float d = 0.0f;
      int extra = -1, it;
      for (it = 0; it < 40; ++it) {
        float T = T0f + d, T2 = T * T;
        float f = (float)c4 * T2 * T2 + kvf * d + (float)c0r;
        float fp = 4.0f * (float)c4 * T2 * T + kvf;
        float dn = d - f / fp;
        if (!(T0f + dn > 0.0f)) dn = 0.5f * T - T0f;
        float step = dn - d;
        d = dn;
        if (extra == 0) break;
        if (extra < 0 && fabsf(step) <= 2e-7f * (T0f + d)) extra = 0;
      }
      double dd = (double)d;
      double T = T0 + dd, T2 = T * T;
      double f = (double)c4 * T2 * T2 + kv * dd + (double)c0r;
      float fp = 4.0f * (float)c4 * (float)(T2 * T) + kvf;
      dd -= f * (double)(1.0f / fp);
      ok = it < 40 && (T0 + dd) > 0.0;
      T1 = T0 + dd;
    }
    if (!ok) atomicAdd(a.status, 1);
  }
  const Real T1r = (Real)T1, T1sq = T1r * T1r;
  Real th;
  if constexpr (sizeof(Real) == 8)
    th = (Real)(T1 * T1 * T1 * T1 / (4.0 * kPi));
  else
    th = T1sq * T1sq * Real(1.0 / (4.0 * kPi));
  const Real S = S0 + th * S1;
  const Real kS = kap * S;

  // ---- Step 5 solve: (1+B1) s1 + Bc s2 = Br,  A1 s1 + (1+Ac) s2 = Ar -------
  const Real Ar = sAQ.total() + th * Ap - kS * Ad;
  const Real Br = sBQ.total() + th * Bp - kS * Bd;
  const Real m11 = B1p, m12 = Bcc, m21 = As1, m22 = Real(1) + Acc;
  const Real det = m11 * m22 - m12 * m21;
  const Real s1 = (Br * m22 - m12 * Ar) / det;
  const Real s2 = (m11 * Ar - m21 * Br) / det;

  // ---- I^{n+1}, quadrature (sec. 3) -----------------------------------------
  KSum<Real> mE, mF[3], mP[6];
  mE.zero();
  for (int i = 0; i < 3; ++i) mF[i].zero();
  for (int i = 0; i < 6; ++i) mP[i].zero();
  for (int m = 0; m < M; ++m) {
    const Real nxm = s_ang[4 * m], nym = s_ang[4 * m + 1], nzm = s_ang[4 * m + 2], Wm = s_ang[4 * m + 3];
    const Real vn = VEL ? nxm * vt[0] + nym * vt[1] + nzm * vt[2] : Real(0);
    const Real rd = fast_rcp(A0 - A1 * vn);
    const Real pe = A1 * (C + Real(3) * vn) * rd;
    const Real rs = s_Q[(size_t)m * L.ncell + tid] + pe * th - kS * rd;   // r'_m
    const Real cm = cq * vn;
    const Real I1 = (rs - s1 - cm * s2) * fast_rcp(a0 - a1 * vn);
    a.I_out[(long long)m * N + c] = I1;
    const Real wi = Wm * I1;
    mE.part += wi;
    const Real wx = nxm * wi, wy = nym * wi, wz = nzm * wi;
    mF[0].part += wx; mF[1].part += wy; mF[2].part += wz;
    mP[0].part += nxm * wx; mP[1].part += nym * wy; mP[2].part += nzm * wz;
    mP[3].part += nym * wx; mP[4].part += nzm * wx; mP[5].part += nzm * wy;
    if ((m & 7) == 7) {
      mE.fold();
      for (int i = 0; i < 3; ++i) mF[i].fold();
      for (int i = 0; i < 6; ++i) mP[i].fold();
    }
  }
  const Real fourpi = Real(4.0 * kPi);
  a.mom_out[c] = fourpi * mE.total();
  Real post[3];
  for (int i = 0; i < 3; ++i) {
    post[i] = mF[i].total();
    a.mom_out[(1 + i) * N + c] = fourpi * post[i];
  }
  for (int i = 0; i < 6; ++i) a.mom_out[(4 + i) * N + c] = fourpi * mP[i].total();

  // ---- gas sources (sec. 4.3: Delta E_T, eqs. momentumchange, kinetichange)
  const Real kmom = -fourpi * a.P * invC;
  Real dEK = 0;
  for (int i = 0; i < 3; ++i) {
    const Real dmom = kmom * (post[i] - pre[i].total());
    a.dMom[i * N + c] = dmom;
    const Real m0 = rho * vin[i];
    dEK += ((m0 + dmom) * (m0 + dmom) - m0 * m0) / (Real(2) * rho);
  }
  a.T_out[c] = T1;
  a.dEgas[c] = kv * (T1 - T0) + (double)dEK;
}

template <typename Real, int DIM, bool VEL>
cudaError_t launch_one(const StepArgs<Real> &a, TileShape t, cudaStream_t s) {
  size_t sm = smem_bytes(DIM, a.M, VEL, t.tx, t.ty, t.tz, sizeof(Real));
  auto kern = step_kernel<Real, DIM, VEL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 block(t.tx, t.ty, t.tz);
  dim3 grid((a.n[0] + t.tx - 1) / t.tx, (a.n[1] + t.ty - 1) / t.ty, (a.n[2] + t.tz - 1) / t.tz);
  kern<<<grid, block, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename Real>
bool choose_tile(int dim, int M, bool has_v, TileShape *out) {
  // preferred shapes (x widest for coalescing), shrunk until they fit
  TileShape cand[4];
  int nc = 0;
  if (dim == 1) {
    cand[nc++] = {512, 1, 1}; cand[nc++] = {256, 1, 1}; cand[nc++] = {128, 1, 1}; cand[nc++] = {64, 1, 1};
  } else if (dim == 2) {
    cand[nc++] = {32, 16, 1}; cand[nc++] = {32, 8, 1}; cand[nc++] = {16, 8, 1}; cand[nc++] = {16, 4, 1};
  } else {
    cand[nc++] = {16, 8, 4}; cand[nc++] = {8, 8, 4}; cand[nc++] = {8, 4, 4}; cand[nc++] = {8, 4, 2};
  }
  const size_t limit = 227 * 1024;
  for (int i = 0; i < nc; ++i) {
    if (smem_bytes(dim, M, has_v, cand[i].tx, cand[i].ty, cand[i].tz, sizeof(Real)) <= limit) {
      *out = cand[i];
      return true;
    }
  }
  return false;
}

template <typename Real>
cudaError_t launch_step(const StepArgs<Real> &a, int dim, bool has_v, TileShape t, cudaStream_t s) {
  if (dim == 1) return has_v ? launch_one<Real, 1, true>(a, t, s) : launch_one<Real, 1, false>(a, t, s);
  if (dim == 2) return has_v ? launch_one<Real, 2, true>(a, t, s) : launch_one<Real, 2, false>(a, t, s);
  return has_v ? launch_one<Real, 3, true>(a, t, s) : launch_one<Real, 3, false>(a, t, s);
}

template bool choose_tile<float>(int, int, bool, TileShape *);
template bool choose_tile<double>(int, int, bool, TileShape *);
template cudaError_t launch_step<float>(const StepArgs<float> &, int, bool, TileShape, cudaStream_t);
template cudaError_t launch_step<double>(const StepArgs<double> &, int, bool, TileShape, cudaStream_t);

}  // namespace rtg
