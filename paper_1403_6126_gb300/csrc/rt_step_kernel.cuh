// Fused radiation-transfer step for sm_103a (Jiang, Stone & Davis 2014,
// arXiv:1403.6126, secs. 3-4): the double-precision kernel (process_tile
// with Real = double) and the tile geometry that the float kernel of
// rt_step_pair.cuh shares.
//
// One CTA owns a tile of cells, one thread per cell, and walks the angles.
// Per angle, in four phases separated by CTA barriers:
//   1. stage I~ = I - IV/C and IV = 3 n.v J of the tile and of a two-cell
//      halo on each active axis (only the cross-shaped part the stencil
//      reads), boundary values applied while staging; the loads of the
//      next angle are issued right after, into registers;
//   2. van Leer slopes, once per cell and axis (own cell along every axis,
//      and the one-layer extension of the tile along its axis);
//   3. one flux per face (the face above the own cell; the tile's lowest
//      face too for cells on the lower edge), pre-multiplied by dt/dx;
//   4. Delta F_m = sum over axes of (flux below - flux above), folded into
//      the right-hand side of the implicit step it belongs to, plus every
//      angle sum of the implicit solves (linear in the stored Q_m).
// After the last angle each thread solves its cell: the T^4 energy equation
// of Step 4 (sec. 4.3) reduced to a scalar quartic, the 2x2 system of Step 5
// (sec. 4.4), then I^{n+1}, the moments E_r, F_r, P_r (sec. 3) and the gas
// sources.  I is read once from and written once to global memory per step.
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
// The Step 4 sums are kept as moments of vn (sum W vn^k / d and
// sum W vn^k r / d, k = 0..3), from which S, J and v.H follow exactly.
#pragma once

#include <math.h>

#include "rt_internal.h"

namespace rtg {

namespace stepk {

constexpr int kHalo = 2;

// Index checking.  A debug build defines RT_BOUNDS_CHECK: every shared- and
// global-memory index of the float step's per-tile code then passes through
// RT_IDX(i, n), and an index outside [0, n) adds one to the step's failure
// count (the same word as a failed temperature solve, so rt_sync reports
// it) and is replaced by 0, which turns an out-of-bounds access into a
// reported error instead of a fault.  In the product build RT_IDX(i, n) is
// i and costs nothing.
__device__ __forceinline__ long long checked_index(long long i, long long n, int *status) {
  if (i >= 0 && i < n) return i;
  atomicAdd(status, 1);
  return 0;
}
#ifdef RT_BOUNDS_CHECK
#define RT_IDX(i, n) (::rtg::stepk::checked_index((i), (n), a.status))
#else
#define RT_IDX(i, n) (i)
#endif
constexpr double kPi = 3.14159265358979323846;

enum { BC_PERIODIC = 0, BC_VACUUM = 1, BC_COPY = 2, BC_INFLOW = 3 };

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

// Half of the van Leer limited slope (Stone & Mihalas 1992, eq. 4): the
// slope is the harmonic mean 2 dl dr / (dl + dr) of the one-sided
// differences when they agree in sign, else 0; half of it, p / (dl + dr),
// is what the face states q +- (1 - nu)/2 * slope need.
template <typename R>
__device__ __forceinline__ R vl_half(R qm, R q0, R qp) {
  R dl = q0 - qm, dr = qp - q0;
  R pr = dl * dr;
  return pr > R(0) ? pr * fast_rcp(dl + dr) : R(0);
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

// Tile geometry shared by host and device.  A tile of T[0] x T[1] x T[2]
// cells (one thread each) is staged with a two-cell halo on every active
// axis; only the cross-shaped part of the padded box is read (the stencil
// moves along one axis at a time), so only the tile cells and the four
// halo layers of each axis are staged ("cross" cells).  Slopes are kept for
// the tile plus one extension layer per axis, face fluxes for the T[d]+1
// faces per axis.
struct Geo {
  int T[3] = {1, 1, 1}, B[3] = {1, 1, 1}, P[3] = {1, 1, 1};   // tile, padded box, cells per layer
  int ncell = 1, nbox = 1, ncross = 1, next = 0, nlow = 0;
  int RX = 1, RXF = 1;          // row lengths of the x slope / flux arrays
  int sl_off[4] = {0, 0, 0, 0}, fx_off[4] = {0, 0, 0, 0};  // slope / flux array offsets per axis
  bool quad = false;            // the layout of the quad kernel (16-byte entries)
  __host__ __device__ constexpr void init(int dim, int tx, int ty, int tz, bool q = false) {
    quad = q;
    T[0] = tx; T[1] = ty; T[2] = tz;
    ncell = tx * ty * tz;
    nbox = 1;
    ncross = ncell;
    next = 0;
    nlow = 0;
    // Threads are ordered x, then z, then y, so a warp holds 32/tx rows of
    // x at consecutive z.  Rows of the x arrays are padded to a length
    // congruent to tx mod 32, which puts those rows on disjoint banks.
    RX = tx >= 32 ? tx + 2 : tx + 32;
    RXF = tx >= 32 ? tx + 1 : tx + 32;
    // The quad kernel's 16-byte entries take eight lanes per shared-memory
    // wavefront.  Its x-halo, x-extension and lowest-x-face work items run
    // along y, so there the box row and the rows of the x arrays (y
    // innermost) have odd lengths: eight items consecutive in y then fall on
    // eight different bank groups.  Tile rows along x are conflict free
    // with any row length.
    if (quad) {
      RX = (tx + 2) | 1;
      RXF = (tx + 1) | 1;
    }
    sl_off[0] = fx_off[0] = 0;
    for (int d = 0; d < 3; ++d) {
      bool act = d < dim;
      B[d] = act ? T[d] + 2 * kHalo : 1;
      if (quad && d == 0 && dim >= 2) B[0] |= 1;
      nbox *= B[d];
      P[d] = ncell / T[d];
      ncross += act ? 2 * kHalo * P[d] : 0;
      next += act ? 2 * P[d] : 0;
      nlow += act ? P[d] : 0;
      sl_off[d + 1] = sl_off[d] + (act ? sl_size(d) : 0);
      fx_off[d + 1] = fx_off[d] + (act ? fx_size(d) : 0);
    }
  }
  // Slope of the cell at local (lx, ly, lz) along axis d, l_d in [-1, T_d].
  __host__ __device__ constexpr int sl_idx(int d, int lx, int ly, int lz) const {
    return d == 0 ? (lx + 1) + RX * (quad ? ly + T[1] * lz : lz + T[2] * ly)
           : d == 1 ? lx + T[0] * (lz + T[2] * (ly + 1))
                    : lx + T[0] * ((lz + 1) + (T[2] + 2) * ly);
  }
  __host__ __device__ constexpr int sl_size(int d) const {
    return d == 0 ? RX * T[2] * T[1] : d == 1 ? T[0] * T[2] * (T[1] + 2) : T[0] * (T[2] + 2) * T[1];
  }
  __host__ __device__ constexpr int sl_step(int d) const { return d == 0 ? 1 : d == 1 ? T[0] * T[2] : T[0]; }
  // Flux of face f along d (between local f-1 and f) in the row of (lx, ly, lz).
  __host__ __device__ constexpr int fx_idx(int d, int f, int lx, int ly, int lz) const {
    return d == 0   ? f + RXF * (quad ? ly + T[1] * lz : lz + T[2] * ly)
           : d == 1 ? lx + T[0] * (lz + T[2] * f)
                    : lx + T[0] * (f + (T[2] + 1) * ly);
  }
  __host__ __device__ constexpr int fx_size(int d) const {
    return d == 0 ? RXF * T[2] * T[1] : d == 1 ? T[0] * T[2] * (T[1] + 1) : T[0] * (T[2] + 1) * T[1];
  }
  __host__ __device__ constexpr int fx_step(int d) const { return d == 0 ? 1 : d == 1 ? T[0] * T[2] : T[0]; }
};

// The same geometry for a compile-time shape, as constants, for device
// code (runtime-indexed member arrays would put the struct in memory).
template <int DIM, int TX, int TY, int TZ, bool Q = false>
struct GeoT {
  __host__ __device__ static constexpr Geo g() {
    Geo x;
    x.init(DIM, TX, TY, TZ, Q);
    return x;
  }
  static constexpr int ncell = g().ncell, nbox = g().nbox, ncross = g().ncross, next = g().next, nlow = g().nlow;
  static constexpr int B0 = g().B[0], B1 = g().B[1];
  static constexpr int P0 = g().P[0], P1 = g().P[1], P2 = g().P[2];
  static constexpr int SL0 = g().sl_off[0], SL1 = g().sl_off[1], SL2 = g().sl_off[2], SL3 = g().sl_off[3];
  static constexpr int FX0 = g().fx_off[0], FX1 = g().fx_off[1], FX2 = g().fx_off[2], FX3 = g().fx_off[3];
  static constexpr int RX = g().RX, RXF = g().RXF;
  __host__ __device__ static constexpr int T(int d) { return d == 0 ? TX : d == 1 ? TY : TZ; }
  __host__ __device__ static constexpr int P(int d) { return d == 0 ? P0 : d == 1 ? P1 : P2; }
  __host__ __device__ static constexpr int bstride(int d) { return d == 0 ? 1 : d == 1 ? B0 : B0 * B1; }
  __host__ __device__ static constexpr int sl_off(int d) { return d == 0 ? SL0 : d == 1 ? SL1 : SL2; }
  __host__ __device__ static constexpr int fx_off(int d) { return d == 0 ? FX0 : d == 1 ? FX1 : FX2; }
  __host__ __device__ static constexpr int sl_idx(int d, int lx, int ly, int lz) {
    return d == 0 ? (lx + 1) + RX * (Q ? ly + TY * lz : lz + TZ * ly)
           : d == 1 ? lx + TX * (lz + TZ * (ly + 1))
                    : lx + TX * ((lz + 1) + (TZ + 2) * ly);
  }
  __host__ __device__ static constexpr int sl_step(int d) { return d == 0 ? 1 : d == 1 ? TX * TZ : TX; }
  __host__ __device__ static constexpr int fx_idx(int d, int f, int lx, int ly, int lz) {
    return d == 0   ? f + RXF * (Q ? ly + TY * lz : lz + TZ * ly)
           : d == 1 ? lx + TX * (lz + TZ * f)
                    : lx + TX * (f + (TZ + 1) * ly);
  }
  __host__ __device__ static constexpr int fx_step(int d) { return d == 0 ? 1 : d == 1 ? TX * TZ : TX; }
};

// Per-angle table entries: n (0-2), W (3), C mu dt/2dx (4-6), C |mu| dt/2dx
// (8-10), mu dt/dx (12-14), W n (16-18).
constexpr int kTab = 20;

// Shared-memory bytes of one CTA: per-angle table (kTab reals per angle), Q
// (M per cell), staged I~ and IV, slopes of both, one flux per face.
__host__ __device__ inline size_t smem_bytes(int dim, int M, bool has_v, int tx, int ty, int tz, size_t rs) {
  Geo g;
  g.init(dim, tx, ty, tz);
  size_t q = has_v ? 2 : 1;
  size_t reals = kTab * (size_t)M + (size_t)M * g.ncell + q * g.nbox + q * g.sl_off[3] + g.fx_off[3];
  return reals * rs + 16;
}

// Maps coordinate g along an axis of n cells onto the grid: the periodic
// image, or the nearest cell for the other boundary kinds.
__device__ __forceinline__ int map_in(int g, int n, int kind_lo, int kind_hi) {
  if (g < 0) return kind_lo == BC_PERIODIC ? ((g % n) + n) % n : 0;
  if (g >= n) return kind_hi == BC_PERIODIC ? g % n : n - 1;
  return g;
}

// Flux through one face, already multiplied by dt/dx: the alpha blend of
// the van Leer states of I~ (sec. 4.2: upwind weight (1+alpha)/2,
// downwind (1-alpha)/2, speed alpha C, written as hc (L+R) + hca alpha (L-R)
// with hc = C mu dt/(2dx), hca = C |mu| dt/(2dx)), plus mu times the IV state
// upwinded by the face velocity (weight wl on the left state).
template <typename Real, bool VEL>
__device__ __forceinline__ Real face_flux(Real qL, Real sL, Real qR, Real sR, Real pL, Real tL, Real pR, Real tR,
                                          Real al, Real hv, Real wl, Real hc, Real hca, Real mud) {
  const Real hl2 = Real(1) - al * (hca + hca);  // 1 - nu, nu = alpha C |mu| dt/dx
  const Real L = qL + hl2 * sL, R = qR - hl2 * sR;
  Real flux = hc * (L + R) + (hca * al) * (L - R);
  if (VEL) {
    const Real Lv = pL + hv * tL, Rv = pR - hv * tR;
    flux += mud * (Rv + wl * (Lv - Rv));
  }
  return flux;
}

// alpha, 1 - |v_face| dt/dx and the left-state weight of the face between
// cells gl and gu (grid coordinates, both inside the grid) along axis d.
template <typename Real, bool VEL>
__device__ __forceinline__ void face_consts(const StepArgs<Real> &a, int d, const int gl[3], const int gu[3], Real *al,
                                            Real *hv, Real *wl) {
  const long long N = a.N;
  const long long cl = gl[0] + (long long)a.n[0] * (gl[1] + (long long)a.n[1] * gl[2]);
  const long long cu = gu[0] + (long long)a.n[0] * (gu[1] + (long long)a.n[1] * gu[2]);
  *al = Real(0.5) * (alpha_of(a.dx[d], a.sa[RT_IDX(cl, N)] + a.ss[RT_IDX(cl, N)]) +
                     alpha_of(a.dx[d], a.sa[RT_IDX(cu, N)] + a.ss[RT_IDX(cu, N)]));
  const Real vf = VEL ? Real(0.5) * (a.v[d * N + RT_IDX(cl, N)] + a.v[d * N + RT_IDX(cu, N)]) : Real(0);
  *hv = Real(1) - (vf < Real(0) ? -vf : vf) * a.dtdx[d];
  *wl = vf > Real(0) ? Real(1) : (vf < Real(0) ? Real(0) : Real(0.5));
}

// Staged cross cells per thread of a tile shape.
__host__ __device__ constexpr int slots_for(int dim, int tx, int ty, int tz) {
  Geo g;
  g.init(dim, tx, ty, tz);
  return (g.ncross + g.ncell - 1) / g.ncell;
}

// One tile of one problem: tile coordinates (tbx, tby, tbz) in units of the
// tile shape, thread tid of TX*TY*TZ (ordered x, then z, then y, see Geo),
// shared memory smem_raw of smem_bytes().  Used by the single-problem
// kernel and by the persistent multi-problem kernel.
template <typename Real, int DIM, bool VEL, int TX, int TY, int TZ>
__device__ __forceinline__ void process_tile(const StepArgs<Real> &a, int tid, int tbx, int tby, int tbz,
                                             unsigned char *smem_raw) {
  constexpr int kSlots = slots_for(DIM, TX, TY, TZ);
  static_assert(kSlots <= 4, "tile halo too large for the staging slots");
  using G = GeoT<DIM, TX, TY, TZ>;
  const int M = a.M;
  const long long N = a.N;
  const int nthr = G::ncell;
  const int org[3] = {tbx * TX, tby * TY, tbz * TZ};
  const int bstride[3] = {1, G::B0, G::B0 * G::B1};

  __syncthreads();   // the previous tile of a persistent CTA is done with shared memory
  Real *s_tab = reinterpret_cast<Real *>(smem_raw);   // [M][kTab]
  Real *s_Q = s_tab + kTab * M;                        // [M][ncell]
  Real *s_It = s_Q + (size_t)M * G::ncell;             // [nbox]
  Real *s_IV = s_It + G::nbox;                         // [nbox]            (VEL)
  Real *s_sI = s_IV + (VEL ? G::nbox : 0);             // slopes of I~
  Real *s_sV = s_sI + G::SL3;                          // slopes of IV      (VEL)
  Real *s_fx = s_sV + (VEL ? G::SL3 : 0);              // face fluxes

  const Real C = a.C, invC = a.invC, dt = a.dt;

  // ---- per-angle table: n, W and the transport factors of each axis, all
  // pre-multiplied by dt/dx so a face flux difference is the change of I
  for (int m = tid; m < M; m += nthr) {
    Real *t = s_tab + kTab * m;
    Real W = a.ang[4 * m + 3];
    for (int d = 0; d < 3; ++d) {
      Real mu = a.ang[4 * m + d];
      Real amu = mu < Real(0) ? -mu : mu;
      t[d] = mu;
      t[4 + d] = Real(0.5) * C * mu * a.dtdx[d];    // (C mu / 2) dt/dx
      t[8 + d] = Real(0.5) * C * amu * a.dtdx[d];   // (C |mu| / 2) dt/dx
      t[12 + d] = mu * a.dtdx[d];                   // mu dt/dx
      t[16 + d] = W * mu;                           // W n
    }
    t[3] = W;
    t[7] = t[11] = t[15] = t[19] = Real(0);
  }

  // ---- own cell ---------------------------------------------------------------
  const int loc[3] = {tid % TX, tid / (TX * TZ), (tid / TX) % TZ};
  const int gx = org[0] + loc[0], gy = org[1] + loc[1], gz = org[2] + loc[2];
  const bool valid = gx < a.n[0] && gy < a.n[1] && gz < a.n[2];
  const long long c = valid ? gx + (long long)a.n[0] * (gy + (long long)a.n[1] * gz) : 0;
  int bo = 0;
  for (int d = 0; d < DIM; ++d) bo += (loc[d] + kHalo) * bstride[d];
  int own_sl[3], own_fx[3];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    own_sl[d] = G::sl_off(d) + G::sl_idx(d, loc[0], loc[1], loc[2]);
    own_fx[d] = G::fx_off(d) + G::fx_idx(d, loc[d], loc[0], loc[1], loc[2]);   // face below the cell
  }

  // ---- staging slots: fixed cross cells of this thread ---------------------
  // slot 0 is always the own cell (tid < ncell).  code: 0 interior, else
  // 1 + 2 axis + side of the boundary the cell lies beyond.
  // bc word of a slot: bit 0 = lies beyond a vacuum or inflow face, bit 1 =
  // inflow, bits 2-3 = axis, bit 4 = upper side
  int sl_box[kSlots], sl_code[kSlots], sl_g[kSlots];
  Real sl_w[kSlots][3];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int k = tid + s * nthr;
    sl_box[s] = -1; sl_code[s] = 0; sl_g[s] = 0;
    sl_w[s][0] = sl_w[s][1] = sl_w[s][2] = Real(0);
    if (k >= G::ncross) continue;
    int b[3] = {0, 0, 0};
    if (k < G::ncell) {
      b[0] = k % TX + (DIM >= 1 ? kHalo : 0);
      b[2] = (k / TX) % TZ + (DIM >= 3 ? kHalo : 0);
      b[1] = k / (TX * TZ) + (DIM >= 2 ? kHalo : 0);
    } else {
      int kk = k - G::ncell;
      int d = 0;
      while (kk >= 2 * kHalo * G::P(d)) { kk -= 2 * kHalo * G::P(d); ++d; }
      int layer = kk / G::P(d), o = kk % G::P(d);
      int side = layer / kHalo, h = layer % kHalo;
      int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      const int bd = side == 0 ? h : G::T(d) + kHalo + h;
      const int b1v = o % G::T(a1) + (a1 < DIM ? kHalo : 0), b2v = o / G::T(a1) + (a2 < DIM ? kHalo : 0);
      b[0] = d == 0 ? bd : (a1 == 0 ? b1v : b2v);
      b[1] = d == 1 ? bd : (a1 == 1 ? b1v : b2v);
      b[2] = d == 2 ? bd : (a1 == 2 ? b1v : b2v);
    }
    sl_box[s] = b[0] + G::B0 * (b[1] + G::B1 * b[2]);
    int g[3], code = 0;
    for (int d = 0; d < 3; ++d) {
      g[d] = d < DIM ? org[d] + b[d] - kHalo : 0;
      if (d < DIM && (g[d] < 0 || g[d] >= a.n[d])) {
        if (code == 0) code = 1 + 2 * d + (g[d] >= a.n[d] ? 1 : 0);
        g[d] = map_in(g[d], a.n[d], a.bc[d][0], a.bc[d][1]);
      }
    }
    if (code) {
      const int axis = (code - 1) >> 1, side = (code - 1) & 1;
      const int kind = a.bc[axis][side];
      code = (kind == BC_VACUUM || kind == BC_INFLOW) ? (1 | (kind == BC_INFLOW ? 2 : 0) | (axis << 2) | (side << 4)) : 0;
    }
    sl_code[s] = code;
    sl_g[s] = (int)(g[0] + (long long)a.n[0] * (g[1] + (long long)a.n[1] * g[2]));
    if (VEL) {
      // w = 3 J v with J = E/(4 pi): IV_m = n_m . w
      const long long cc = sl_g[s];
      const Real w3 = Real(3.0 / (4.0 * kPi)) * a.mom_in[cc];
      sl_w[s][0] = w3 * a.v[cc];
      sl_w[s][1] = w3 * a.v[N + cc];
      sl_w[s][2] = w3 * a.v[2 * N + cc];
    }
  }

  // ---- slope-extension items of this thread (at most two: next <= 2 ncell)
  int ext_bb[2] = {0, 0}, ext_st[2] = {0, 0}, ext_si[2] = {-1, -1};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int e = tid + j * nthr;
    if (e >= G::next) continue;
    int ee = e, d = 0;
    while (ee >= 2 * G::P(d)) { ee -= 2 * G::P(d); ++d; }
    const int side = ee / G::P(d), o = ee % G::P(d);
    const int a1x = d == 0 ? 1 : 0, a2x = d == 2 ? 1 : 2;
    const int ld = side == 0 ? -1 : G::T(d), l1v = o % G::T(a1x), l2v = o / G::T(a1x);
    const int l0 = d == 0 ? ld : (a1x == 0 ? l1v : l2v);
    const int l1 = d == 1 ? ld : (a1x == 1 ? l1v : l2v);
    const int l2 = d == 2 ? ld : (a1x == 2 ? l1v : l2v);
    ext_bb[j] = (l0 + kHalo) + G::B0 * ((DIM >= 2 ? l1 + kHalo : 0) + G::B1 * (DIM >= 3 ? l2 + kHalo : 0));
    ext_st[j] = G::bstride(d);
    ext_si[j] = G::sl_off(d) + G::sl_idx(d, l0, l1, l2);
  }
  const int ncell = G::ncell;

  // ---- face constants.  alpha of a face is the mean of its two cells'; the
  // IV face blends the van Leer states by the sign of the face velocity
  // (weight wl of the left state); hv = 1 - |v_face| dt/dx.
  // Upper face of each axis of the own cell: registers.
  Real fu_al[3], fu_hv[3], fu_wl[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) { fu_al[d] = Real(1); fu_hv[d] = Real(1); fu_wl[d] = Real(0.5); }
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    int gl[3] = {min(gx, a.n[0] - 1), min(gy, a.n[1] - 1), min(gz, a.n[2] - 1)};
    int gu[3] = {gl[0], gl[1], gl[2]};
    gu[d] = map_in((d == 0 ? gx : d == 1 ? gy : gz) + 1, a.n[d], a.bc[d][0], a.bc[d][1]);
    face_consts<Real, VEL>(a, d, gl, gu, &fu_al[d], &fu_hv[d], &fu_wl[d]);
  }
  // The lowest face of the tile along each axis: work items spread over the
  // threads (at most two each), so no warp diverges over them.
  int lf_d[2] = {0, 0}, lf_bb[2] = {0, 0}, lf_si[2] = {0, 0}, lf_sstep[2] = {1, 1}, lf_fx[2] = {-1, -1};
  Real lf_al[2] = {1, 1}, lf_hv[2] = {1, 1}, lf_wl[2] = {0.5, 0.5};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    int e = tid + j * nthr;
    if (e >= G::nlow) continue;
    int d = 0;
    while (e >= G::P(d)) { e -= G::P(d); ++d; }
    const int a1x = d == 0 ? 1 : 0;
    const int l1v = e % G::T(a1x), l2v = e / G::T(a1x);
    const int l[3] = {d == 0 ? 0 : (a1x == 0 ? l1v : l2v), d == 1 ? 0 : (a1x == 1 ? l1v : l2v),
                      d == 2 ? 0 : (a1x == 2 ? l1v : l2v)};
    const int bb = (l[0] + kHalo) + G::B0 * ((DIM >= 2 ? l[1] + kHalo : 0) + G::B1 * (DIM >= 3 ? l[2] + kHalo : 0));
    const int st = G::bstride(d);
    lf_d[j] = d;
    lf_bb[j] = bb - st;                                    // cell below the face
    lf_si[j] = G::sl_off(d) + G::sl_idx(d, d == 0 ? -1 : l[0], d == 1 ? -1 : l[1], d == 2 ? -1 : l[2]);   // slope below
    lf_sstep[j] = G::sl_step(d);
    lf_fx[j] = G::fx_off(d) + G::fx_idx(d, 0, l[0], l[1], l[2]);   // face 0 of this row
    int gu[3] = {min(org[0] + l[0], a.n[0] - 1), min(org[1] + (DIM >= 2 ? l[1] : 0), a.n[1] - 1),
                 min(org[2] + (DIM >= 3 ? l[2] : 0), a.n[2] - 1)};
    int gl[3] = {gu[0], gu[1], gu[2]};
    const int od = d == 0 ? org[0] : d == 1 ? org[1] : org[2], nd = d == 0 ? a.n[0] : d == 1 ? a.n[1] : a.n[2];
    const int kl = d == 0 ? a.bc[0][0] : d == 1 ? a.bc[1][0] : a.bc[2][0], kh = d == 0 ? a.bc[0][1] : d == 1 ? a.bc[1][1] : a.bc[2][1];
    const int gud = min(od, nd - 1), gld = map_in(od - 1, nd, kl, kh);
    if (d == 0) { gu[0] = gud; gl[0] = gld; } else if (d == 1) { gu[1] = gud; gl[1] = gld; } else { gu[2] = gud; gl[2] = gld; }
    face_consts<Real, VEL>(a, d, gl, gu, &lf_al[j], &lf_hv[j], &lf_wl[j]);
  }

  // ---- per-cell constants of the implicit steps ------------------------------
  Real rho = 1, sa = 0, ss = 0, vt[3] = {0, 0, 0}, vin[3] = {0, 0, 0};
  double T0 = 1.0;
  if (valid) {
    rho = a.rho[c]; sa = a.sa[c]; ss = a.ss[c];
    T0 = a.T_in[c];
    if (VEL) {
      for (int d = 0; d < 3; ++d) vin[d] = a.v[d * N + c];
      if (a.estimate_v) {
        // Step 3 (sec. 4.5): per axis, backward-Euler momentum exchange with
        // E, F, P_dd held at their step-n values
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
  const Real to_scat = ss > sa ? Real(1) : Real(0);
  const Real v2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
  const Real A0 = Real(1) + dt * C * sa, A1 = dt * sa, kap = dt * sa / C;
  const Real a0 = Real(1) + dt * C * ss, a1 = dt * ss;
  const Real bq0 = -dt * C * ss - dt * ss * v2 / C, bq1 = Real(2) * dt * ss, bq2 = -dt * ss / C;
  const Real cq = Real(-3) * dt * ss;
  const Real apb0 = Real(1) - a1 * v2 * invC, apb2 = -a1 * invC;
  // without velocity terms the reciprocals are per-cell constants
  const Real rd0 = VEL ? Real(0) : fast_rcp(A0);
  const Real ra0 = VEL ? Real(0) : fast_rcp(a0);

  // Step 4 sums in powers of vn = n.v~: T_k = sum W vn^k / d, U_k = sum W vn^k r / d
  Real T0s = 0, T1s = 0, T2s = 0, T3s = 0;
  KSum<Real> U0; U0.zero();
  Real U1 = 0, U2 = 0;
  // Step 5 sums (1/a = W / a')
  KSum<Real> AQ; AQ.zero();
  Real Ap = 0, Ad = 0, As1 = 0, Acc = 0, BQ = 0, Bp = 0, Bd = 0, B1p = 0, Bcc = 0;
  Real pre0 = 0, pre1 = 0, pre2 = 0;   // sum W n (I^n + Delta F)

  // prefetch angle 0
  Real pf[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) pf[s] = sl_box[s] >= 0 ? a.I_in[sl_g[s]] : Real(0);
  const Real *I_next = a.I_in;
  __syncthreads();

  for (int m = 0; m < M; ++m) {
    const Real *t = s_tab + kTab * m;
    const Real nxm = t[0], nym = t[1], nzm = t[2], Wm = t[3];
    // ---- phase 1: stage I~ = I - IV/C and IV of the cross cells -------------
    Real I0 = 0, q0 = 0, p0 = 0;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      if (sl_box[s] < 0) continue;
      Real I = pf[s];
      if (sl_code[s]) {
        const int axis = (sl_code[s] >> 2) & 3, side = (sl_code[s] >> 4) & 1;
        const Real mu = t[axis];
        const bool incoming = side ? (mu < Real(0)) : (mu > Real(0));
        if (incoming) I = (sl_code[s] & 2) ? a.inflow[(axis * 2 + side) * M + m] : Real(0);
      }
      Real IV = 0, It = I;
      if (VEL) {
        IV = nxm * sl_w[s][0] + nym * sl_w[s][1] + nzm * sl_w[s][2];
        It = I - IV * invC;
        s_IV[sl_box[s]] = IV;
      }
      s_It[sl_box[s]] = It;
      if (s == 0) { I0 = I; q0 = It; p0 = IV; }
    }
    if (m + 1 < M) {
      I_next += N;
#pragma unroll
      for (int s = 0; s < kSlots; ++s)
        if (sl_box[s] >= 0) pf[s] = I_next[sl_g[s]];
    }
    __syncthreads();

    // ---- phase 2: van Leer slopes (half slopes p/(dl+dr)) of own cell along
    // every axis, and of the extension cells along their axis -------------
    Real sI[3], sV[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int st = bstride[d];
      sI[d] = vl_half(s_It[bo - st], q0, s_It[bo + st]);
      s_sI[own_sl[d]] = sI[d];
      if (VEL) {
        sV[d] = vl_half(s_IV[bo - st], p0, s_IV[bo + st]);
        s_sV[own_sl[d]] = sV[d];
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (ext_si[j] < 0) continue;
      const int bb = ext_bb[j], st = ext_st[j];
      s_sI[ext_si[j]] = vl_half(s_It[bb - st], s_It[bb], s_It[bb + st]);
      if (VEL) s_sV[ext_si[j]] = vl_half(s_IV[bb - st], s_IV[bb], s_IV[bb + st]);
    }
    __syncthreads();

    // ---- phase 3: face fluxes (pre-multiplied by dt/dx) -------------------
    Real fhi[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int st = bstride[d];
      const Real hc = t[4 + d], hca = t[8 + d], mud = t[12 + d];
      // face above the own cell
      const int sn = own_sl[d] + G::sl_step(d);
      fhi[d] = face_flux<Real, VEL>(q0, sI[d], s_It[bo + st], s_sI[sn], p0, VEL ? sV[d] : Real(0),
                                    VEL ? s_IV[bo + st] : Real(0), VEL ? s_sV[sn] : Real(0),
                                    fu_al[d], fu_hv[d], fu_wl[d], hc, hca, mud);
      s_fx[own_fx[d] + G::fx_step(d)] = fhi[d];
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (lf_fx[j] < 0) continue;
      const int d = lf_d[j], bb = lf_bb[j], st = d == 0 ? 1 : bstride[d == 1 ? 1 : 2];
      const int si = lf_si[j], si1 = lf_si[j] + lf_sstep[j];
      s_fx[lf_fx[j]] = face_flux<Real, VEL>(s_It[bb], s_sI[si], s_It[bb + st], s_sI[si1],
                                            VEL ? s_IV[bb] : Real(0), VEL ? s_sV[si] : Real(0),
                                            VEL ? s_IV[bb + st] : Real(0), VEL ? s_sV[si1] : Real(0),
                                            lf_al[j], lf_hv[j], lf_wl[j], t[4 + d], t[8 + d], t[12 + d]);
    }
    __syncthreads();

    // ---- phase 4: Delta F_m, right-hand sides and the angle sums ----------
    Real dF = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) dF += s_fx[own_fx[d]] - fhi[d];
    const Real full = I0 + dF;
    Real vn = 0, rd = rd0, ra = ra0;
    if (VEL) {
      vn = nxm * vt[0] + nym * vt[1] + nzm * vt[2];
      rd = fast_rcp(A0 - A1 * vn);
      ra = fast_rcp(a0 - a1 * vn);
    }
    const Real qa = (to_scat > Real(0) ? I0 : full) * rd;   // r_m / d_m
    const Real Q = qa + to_scat * dF;
    s_Q[(size_t)m * ncell + tid] = Q;
    const Real wrd = Wm * rd;
    const Real wq = Wm * qa;
    T0s += wrd; U0.part += wq;
    if (VEL) {
      const Real x1 = wrd * vn, x2 = x1 * vn;
      T1s += x1; T2s += x2; T3s += x2 * vn;
      const Real y1 = wq * vn;
      U1 += y1; U2 += y1 * vn;
    }
    const Real pe = A1 * (C + Real(3) * vn) * rd;          // e_m / d_m
    const Real wa = Wm * ra;                               // 1 / a_m
    AQ.part += wa * Q; Ap += wa * pe; Ad += wa * rd; As1 += wa;
    if (VEL) {
      const Real bm = bq0 + vn * (bq1 + bq2 * vn);
      const Real cm = cq * vn;
      const Real bwa = bm * wa;
      Acc += cm * wa;
      BQ += bwa * Q; Bp += bwa * pe; Bd += bwa * rd; Bcc += cm * bwa;
      B1p += wa * (apb0 + vn * (a1 + apb2 * vn));
    } else {
      const Real bwa = bq0 * wa;
      BQ += bwa * Q; Bp += bwa * pe; Bd += bwa * rd;
      B1p += wa;
    }
    pre0 += t[16] * full; pre1 += t[17] * full; pre2 += t[18] * full;
    if ((m & 7) == 7) { U0.fold(); AQ.fold(); }
  }

  if (!valid) return;

  // ---- Step 4 solve: S, J, v.H affine in theta; scalar quartic in T ---------
  const Real Wr = U0.total(), Vr = U1, Gr = v2 * Wr + U2;
  const Real W1 = T0s, V1 = T1s, G1 = v2 * T0s + T2s;
  const Real We = A1 * (C * T0s + Real(3) * T1s);
  const Real Ve = A1 * (C * T1s + Real(3) * T2s);
  const Real Ge = A1 * (C * (v2 * T0s + T2s) + Real(3) * (v2 * T1s + T3s));
  const Real Wq = T0s - Real(4) * A1 * T1s;     // sum W (d - e) / d
  (void)We;
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
      // the FP64 reference's iteration and stopping rule (with its default
      // options): Newton from T^n until |dT| <= newton_rtol T, then one more
      // step, at most newton_max_it steps
      const double c0 = (double)c0r - kv * T0, c4d = (double)c4;
      const double rtol = a.newton_rtol;
      const int max_it = a.newton_max_it;
      double T = T0;
      int extra = -1, it;
      for (it = 0; it < max_it; ++it) {
        double T3 = T * T * T;
        double f = c4d * T3 * T + kv * T + c0;
        double fp = 4.0 * c4d * T3 + kv;
        double Tn = T - f / fp;
        if (!(Tn > 0)) Tn = 0.5 * T;
        double dT = Tn - T;
        T = Tn;
        if (extra == 0) break;
        if (extra < 0 && fabs(dT) <= rtol * T) extra = 0;
      }
      ok = it < max_it;
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
  const Real Ar = AQ.total() + th * Ap - kS * Ad;
  const Real Br = BQ + th * Bp - kS * Bd;
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
    const Real *t = s_tab + kTab * m;
    const Real nxm = t[0], nym = t[1], nzm = t[2], Wm = t[3];
    Real vn = 0, rd = rd0, ra = ra0;
    if (VEL) {
      vn = nxm * vt[0] + nym * vt[1] + nzm * vt[2];
      rd = fast_rcp(A0 - A1 * vn);
      ra = fast_rcp(a0 - a1 * vn);
    }
    const Real pe = A1 * (C + Real(3) * vn) * rd;
    const Real rs = s_Q[(size_t)m * ncell + tid] + pe * th - kS * rd;   // r'_m
    const Real cm = cq * vn;
    const Real I1 = (rs - s1 - cm * s2) * ra;
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
  const Real pre[3] = {pre0, pre1, pre2};
  for (int i = 0; i < 3; ++i) {
    const Real dmom = kmom * (post[i] - pre[i]);
    a.dMom[i * N + c] = dmom;
    const Real m0 = rho * vin[i];
    dEK += ((m0 + dmom) * (m0 + dmom) - m0 * m0) / (Real(2) * rho);
  }
  a.T_out[c] = T1;
  a.dEgas[c] = kv * (T1 - T0) + (double)dEK;
}

template <typename Real, int DIM, bool VEL, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ) step_kernel(const StepArgs<Real> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int o = a.outer_begin;
  process_tile<Real, DIM, VEL, TX, TY, TZ>(a, threadIdx.x, blockIdx.x + (DIM == 1 ? o : 0),
                                           blockIdx.y + (DIM == 2 ? o : 0), blockIdx.z + (DIM == 3 ? o : 0), smem_raw);
}

template <typename Real, int DIM, bool VEL, int TX, int TY, int TZ>
cudaError_t launch_shape(const StepArgs<Real> &a, cudaStream_t s) {
  const size_t sm = smem_bytes(DIM, a.M, VEL, TX, TY, TZ, sizeof(Real));
  auto kern = step_kernel<Real, DIM, VEL, TX, TY, TZ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 block(TX * TY * TZ);
  dim3 grid((a.n[0] + TX - 1) / TX, (a.n[1] + TY - 1) / TY, (a.n[2] + TZ - 1) / TZ);
  if (a.outer_count > 0) (DIM == 3 ? grid.z : DIM == 2 ? grid.y : grid.x) = a.outer_count;
  kern<<<grid, block, sm, s>>>(a);
  return cudaGetLastError();
}

// Shapes compiled for one precision and dimension, preferred first.
template <typename Real, int DIM>
struct Shapes;

// Whether shape t of the list can run M angles: shared memory within the
// opt-in limit (the halo's staging slots are checked at compile time).
inline bool shape_fits(int dim, int M, bool has_v, TileShape t, size_t rs) {
  return smem_bytes(dim, M, has_v, t.tx, t.ty, t.tz, rs) <= 227 * 1024;
}

}  // namespace stepk

}  // namespace rtg
