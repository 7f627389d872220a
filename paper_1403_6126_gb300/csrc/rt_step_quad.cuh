// Fused radiation-transfer step with float intensities in a quad-interleaved
// layout (Jiang, Stone & Davis 2014, arXiv:1403.6126, secs. 3-4).
//
// Storage.  The intensity of a float context is kept as Q = ceil(M/4) planes
// of float4: I[q][c] holds angles 4q .. 4q+3 of cell c (angles past M are
// zero padding).  A thread reads or writes the four angles of its cell with
// one 128-bit access, and the 8 x-consecutive cells of a tile row cover one
// whole 128-byte line.
//
// Same method, tile geometry and reading of the paper as process_tile2
// (rt_step_pair.cuh): one thread per cell, every per-angle quantity carried
// as a pair of angles in packed FP32, four phases per angle quad separated by
// three CTA barriers (stage I~ = I - IV/C and IV, van Leer half slopes, one
// flux per face, Delta F).  The work is split differently:
//  * Transport loop (the phases with barriers): per pair only Delta F_m is
//    formed and written to the output array, two pairs per 128-bit store; no
//    implicit-step quantity lives in these registers.
//  * Source loop (no barriers): reads I^n and Delta F back (both L2 resident:
//    the tile read them microseconds before), forms the right-hand sides Q_m
//    of the implicit step that Delta F belongs to (sec. 4.2: the larger
//    opacity) and overwrites Delta F with Q_m, and takes every angle sum of
//    Steps 4 and 5 in one pass (the intensity sums and the sums that depend
//    only on the velocity and the opacities).
//  * Per-cell solve (the scalar T^4 equation of sec. 4.3 and the 2x2 system
//    of sec. 4.4), then the final loop writes I^{n+1} over Q_m and takes the
//    quadrature of sec. 3.
// The per-pair constants come from a table in the launch parameters (the
// constant bank: warp-uniform loads that use neither shared memory nor its
// bandwidth) when TAB_PARAM is set, else from shared memory (the persistent
// multi-problem kernel, whose problems each have their own table).
//
// Precision.  Every per-angle quantity of the implicit steps is carried as a
// deviation from the cell's center R, its smallest intensity over angles
// (written by the step that produced I^n, or formed from I^n where no such
// array is given), so that 0 <= I_m - R <= I_m: Steps 4 and 5 solve for the
// deviations of theta and of J'' from R, and the moments are R times the
// angle table's own sums plus sums of deviations.  Float rounding then
// scales with the spread of I over angle rather than with I, and never
// exceeds that of I itself.  All angle sums are over the weights normalised to sum 1
// exactly (the float weights sum to 1 + O(1e-8)), so isotropic equilibrium
// stays a fixed point of the energy exchange.  Moments E, F, P and the
// momentum source are written in double.
#pragma once

#include "rt_step_pair.cuh"

namespace rtg {

namespace stepk {

// Pairs a launch-parameter table can hold: 40 (80 angles) for the
// single-problem kernels, 128 (256 angles) for the allocation-free step.
constexpr int kQTabPairsSmall = 40;
constexpr int kQTabPairsLarge = 128;

// Launch-parameter table: the kTab2 entries of every angle (see kTab2),
// interleaved by quad: e[kTab2 q + j] holds entry j of angles 4q .. 4q+3
// (the pair 2q in x, y and the pair 2q + 1 in z, w), so one 128-bit load
// gives an entry for both pairs of a quad; angles past M are zeros
// (weightless, motionless).  Then the inflow intensities [6][2P] per face
// (zero for angles past M).  P, the pairs it holds, is even.
template <int P>
struct QTable {
  float4 e[P / 2 * kTab2];
  float inflow[6][2 * P];
};

// Host side: the table entries exactly as the device would form them (the
// same float products in the same order), so that kernels reading either
// table give bitwise the same result.  ang: [M][4] floats (n_x, n_y, n_z, W);
// inflow: [6][M] floats or NULL.
template <int P>
inline void fill_qtable(QTable<P> *t, const float *ang, int M, float C, const float dtdx[3], const float *inflow) {
  for (int i = 0; i < P / 2 * kTab2; ++i) t->e[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int f = 0; f < 6; ++f)
    for (int m = 0; m < 2 * P; ++m) t->inflow[f][m] = (inflow && m < M) ? inflow[f * M + m] : 0.0f;
  for (int m = 0; m < M && m < 2 * P; ++m) {
    const int q = m / 4, c = m % 4;
    const float W = ang[4 * m + 3];
    for (int j = 0; j < kTab2; ++j) {
      float val;
      if (j < 3) {
        val = ang[4 * m + j];
      } else if (j == 3) {
        val = W;
      } else {
        const int d = (j - 4) % 3, kind = (j - 4) / 3;
        const float mu = ang[4 * m + d], amu = mu < 0.0f ? -mu : mu;
        const float hC = 0.5f * C;
        val = kind == 0   ? hC * mu * dtdx[d]
              : kind == 1 ? hC * amu * dtdx[d]
              : kind == 2 ? mu * dtdx[d]
                          : W * mu;
      }
      float4 &e = t->e[kTab2 * q + j];
      (c == 0 ? e.x : c == 1 ? e.y : c == 2 ? e.z : e.w) = val;
    }
  }
}

// Shared memory of one CTA of the quad kernel: the float4 staging arrays
// (I~, IV, the slopes of I~, one flux per face), plus the pair table when it
// is not a launch parameter.
__host__ __device__ inline size_t smem_bytes_q(int dim, int M, bool has_v, int tx, int ty, int tz, bool tab_param) {
  Geo g;
  g.init(dim, tx, ty, tz, true);
  const size_t q = has_v ? 2 : 1, pairs = 2 * (size_t)((M + 3) / 4);
  const size_t n4 = q * g.nbox + g.sl_off[3] + g.fx_off[3];
  return (tab_param ? 0 : kTab2 * pairs * sizeof(f2)) + n4 * sizeof(float4) + 16;
}

// Exact float -> double by bit assembly (integer pipe: the FP64 pipe is the
// scarce one on this GPU).  Subnormal floats (below 1.2e-38) give 0.
__device__ __forceinline__ double f2d_exact(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xfffffu);
  const unsigned lo = b << 29;
  return e == 0u ? 0.0 : __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ f2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 mk4(f2 a, f2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// IV state of two angles at a face, from the upwind cell alone (sec. 4.2:
// IV is carried at the flow velocity, upwinded by the face velocity): b is
// the upwind cell's slot in the staged box, st the axis stride, sgn = +h
// when the upwind cell lies below the face (its upper van Leer state) and
// -h when above (its lower state), with h = 1 - |v_face| dt / dx.
__device__ __forceinline__ f2 iv_state(const f2 *s_IV, int b, int st, float sgn) {
  const f2 q = s_IV[b];
  return p_fma(dup(sgn), vl_half2(s_IV[b - st], q, s_IV[b + st]), q);
}

// The same for the four angles of a quad (staged as float4).
__device__ __forceinline__ float4 iv_state4(const float4 *s_IV4, int b, int st, float sgn) {
  const float4 qm = s_IV4[b - st], q = s_IV4[b], qp = s_IV4[b + st];   // callers check b - st .. b + st
  return mk4(p_fma(dup(sgn), vl_half2(lo2(qm), lo2(q), lo2(qp)), lo2(q)),
             p_fma(dup(sgn), vl_half2(hi2(qm), hi2(q), hi2(qp)), hi2(q)));
}

// The IV state at a face whose velocity is exactly zero: the mean of the two
// cells' states (lower cell b, upper cell b + st).
__device__ __forceinline__ f2 iv_state_mean(const f2 *s_IV, int b, int st, float h) {
  return p_mul(dup(0.5f), p_add(iv_state(s_IV, b, st, h), iv_state(s_IV, b + st, st, -h)));
}

// Double -> float rounded to nearest (ties to even), by bit assembly on the
// integer pipe.  Results below the float normal range give a signed zero.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int fe = (int)((hi >> 20) & 0x7ffu) - 896;   // the float's biased exponent
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
  const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ? 1u : 0u;
  const unsigned sign = hi & 0x80000000u;
  return fe <= 0 ? __uint_as_float(sign) : __uint_as_float(sign | (((unsigned)fe << 23) + mant + up));
}

// 4 pi times a float pair (hi - lo), as a double: the products with the
// float-float 4 pi are formed in float, exactly enough that the double
// carries the value to ~1e-14 (one FP64 add).
__device__ __forceinline__ double ksum_4pi_double(const KSum2 &s) {
  constexpr float c_h = float(4.0 * kPi);
  constexpr float c_l = float(4.0 * kPi - (double)float(4.0 * kPi));
  const float p = c_h * s.hi;
  const float e = fmaf(c_l, s.hi, fmaf(-c_h, s.lo, fmaf(c_h, s.hi, -p)));
  return f2d_exact(p) + f2d_exact(e);
}

// 4 pi (R s + D) as a double, for a table sum s = sh + sl (float pair) and a
// sum of deviations D: the product R sh is split exactly by an FMA, and the
// remainder R sl + D, the size of the deviations, is formed in float.
__device__ __forceinline__ double mom_4pi_double(float R, float sh, float sl, float D) {
  const float p = R * sh;
  const float t = fmaf(R, sl, fmaf(R, sh, -p)) + D;
  KSum2 k;
  k.hi = p;
  k.lo = -t;
  return ksum_4pi_double(k);
}

template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

template <int DIM, bool VEL, int TX, int TY, int TZ, bool TAB_PARAM, int TP>
__device__ __forceinline__ void process_tile_q(const StepArgs<float> &a, const QTable<TP> *qt, int tid, int tbx,
                                               int tby, int tbz, unsigned char *smem_raw) {
  using G = GeoT<DIM, TX, TY, TZ, true>;
  constexpr int nthr = G::ncell;
  constexpr int kSlots = slots_for(DIM, TX, TY, TZ);
  constexpr int kExt = (G::next + nthr - 1) / nthr;
  constexpr int kLow = (G::nlow + nthr - 1) / nthr;
  static_assert(kSlots <= 4 && kExt <= 2 && kLow <= 2, "tile halo too large for the per-thread work items");
  // slot s holds a staged cell for every thread of the tile
  auto slot_full = [](int s) { return (s + 1) * nthr <= G::ncross; };
  const int M = a.M, NQ = (M + 3) / 4;
  const long long N = a.N;
  const int org[3] = {tbx * TX, tby * TY, tbz * TZ};
  const int bstride[3] = {1, G::B0, G::B0 * G::B1};

  __syncthreads();   // the previous tile of a persistent CTA is done with shared memory
  float4 *s_tab = reinterpret_cast<float4 *>(smem_raw);  // [NQ][kTab2] as QTable::e (shared table only)
  // staging arrays, one float4 (the four angles of a quad) per entry
  float4 *s_It4 = s_tab + (TAB_PARAM ? 0 : kTab2 * NQ);  // I~ [nbox]
  float4 *s_IV4 = s_It4 + G::nbox;                       // IV [nbox] (VEL)
  float4 *s_sI4 = s_IV4 + (VEL ? G::nbox : 0);           // half slopes of I~
  float4 *s_fx4 = s_sI4 + G::SL3;                        // face fluxes
  const float4 *I4 = reinterpret_cast<const float4 *>(a.I_in);
  // entry j of the four angles of quad q
  auto tab4 = [&](int q, int j) -> float4 {
    if constexpr (TAB_PARAM)
      return qt->e[kTab2 * q + j];
    else
      return s_tab[kTab2 * q + j];
  };
  auto inflow = [&](int face, int m) -> float {
    if constexpr (TAB_PARAM)
      return qt->inflow[face][m];
    else
      return m < M ? a.inflow[face * M + m] : 0.0f;
  };

  const float C = a.C, invC = a.invC, dt = a.dt;

  // ---- shared pair table (as fill_qtable) --------------------------------------
  if constexpr (!TAB_PARAM) {
    for (int i = tid; i < kTab2 * NQ; i += nthr) {
      const int q = i / kTab2, j = i % kTab2;
      float v[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int m = 4 * q + h;
        float val = 0.0f;
        if (m < M) {
          const float W = a.ang[4 * m + 3];
          if (j < 3) {
            val = a.ang[4 * m + j];
          } else if (j == 3) {
            val = W;
          } else {
            const int d = (j - 4) % 3, kind = (j - 4) / 3;
            const float mu = a.ang[4 * m + d], amu = mu < 0.0f ? -mu : mu;
            const float hC = 0.5f * C;
            val = kind == 0   ? hC * mu * a.dtdx[d]
                  : kind == 1 ? hC * amu * a.dtdx[d]
                  : kind == 2 ? mu * a.dtdx[d]
                              : W * mu;
          }
        }
        v[h] = val;
      }
      s_tab[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
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
    own_fx[d] = G::fx_off(d) + G::fx_idx(d, loc[d], loc[0], loc[1], loc[2]);
  }

  // ---- staging slots (see process_tile) ---------------------------------------
  int sl_box[kSlots], sl_code[kSlots], sl_g[kSlots];
  float sl_w[kSlots][3];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int k = tid + s * nthr;
    sl_box[s] = -1; sl_code[s] = 0; sl_g[s] = 0;
    sl_w[s][0] = sl_w[s][1] = sl_w[s][2] = 0.0f;
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
      // the x halo hands out its four layers fastest: the two cells of a
      // side share a 32-byte sector of the intensity array, so the loads of
      // eight consecutive items fill four sectors instead of eight
      const int layer = d == 0 ? kk % (2 * kHalo) : kk / G::P(d), o = d == 0 ? kk / (2 * kHalo) : kk % G::P(d);
      const int side = layer / kHalo, h = layer % kHalo;
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
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
      const long long cc = sl_g[s];
      const float w3 = float(3.0 / (4.0 * kPi)) * d2f_rn(a.mom_in[RT_IDX(cc, N)]);
      sl_w[s][0] = w3 * a.v[RT_IDX(cc, N)];
      sl_w[s][1] = w3 * a.v[N + RT_IDX(cc, N)];
      sl_w[s][2] = w3 * a.v[2 * N + RT_IDX(cc, N)];
    }
  }

  // ---- slope-extension items (see process_tile) -------------------------------
  int ext_bb[kExt > 0 ? kExt : 1], ext_st[kExt > 0 ? kExt : 1], ext_si[kExt > 0 ? kExt : 1];
#pragma unroll
  for (int j = 0; j < kExt; ++j) {
    ext_bb[j] = 0; ext_st[j] = 0; ext_si[j] = -1;
    const int e = tid + j * nthr;
    if (e >= G::next) continue;
    int ee = e, d = 0;
    while (ee >= 2 * G::P(d)) { ee -= 2 * G::P(d); ++d; }
    const int side = ee / G::P(d), o = ee % G::P(d);
    const int a1x = d == 0 ? 1 : 0;
    const int ld = side == 0 ? -1 : G::T(d), l1v = o % G::T(a1x), l2v = o / G::T(a1x);
    const int l0 = d == 0 ? ld : (a1x == 0 ? l1v : l2v);
    const int l1 = d == 1 ? ld : (a1x == 1 ? l1v : l2v);
    const int l2 = d == 2 ? ld : (a1x == 2 ? l1v : l2v);
    ext_bb[j] = (l0 + kHalo) + G::B0 * ((DIM >= 2 ? l1 + kHalo : 0) + G::B1 * (DIM >= 3 ? l2 + kHalo : 0));
    ext_st[j] = G::bstride(d);
    ext_si[j] = G::sl_off(d) + G::sl_idx(d, l0, l1, l2);
  }

  // ---- face constants (see process_tile) ---------------------------------------
  float fu_al[3], fu_hv[3], fu_wl[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) { fu_al[d] = 1.0f; fu_hv[d] = 1.0f; fu_wl[d] = 0.5f; }
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    int gl[3] = {min(gx, a.n[0] - 1), min(gy, a.n[1] - 1), min(gz, a.n[2] - 1)};
    int gu[3] = {gl[0], gl[1], gl[2]};
    gu[d] = map_in((d == 0 ? gx : d == 1 ? gy : gz) + 1, a.n[d], a.bc[d][0], a.bc[d][1]);
    face_consts<float, VEL>(a, d, gl, gu, &fu_al[d], &fu_hv[d], &fu_wl[d]);
  }
  // the upper face's upwind cell for IV: offset of its slot from the own
  // cell's (0 below the face, one stride above), the state's sign, and
  // whether the face velocity is exactly zero (mean of both states)
  int iv_off[3] = {0, 0, 0};
  float iv_sg[3] = {1.0f, 1.0f, 1.0f};
  bool iv_mean[3] = {false, false, false};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    iv_off[d] = fu_wl[d] >= 0.5f ? 0 : bstride[d];
    iv_sg[d] = fu_wl[d] >= 0.5f ? fu_hv[d] : -fu_hv[d];
    iv_mean[d] = fu_wl[d] == 0.5f;
  }
  int lf_d[kLow > 0 ? kLow : 1], lf_bb[kLow > 0 ? kLow : 1], lf_si[kLow > 0 ? kLow : 1],
      lf_sstep[kLow > 0 ? kLow : 1], lf_fx[kLow > 0 ? kLow : 1];
  float lf_al[kLow > 0 ? kLow : 1], lf_hv[kLow > 0 ? kLow : 1], lf_wl[kLow > 0 ? kLow : 1];
#pragma unroll
  for (int j = 0; j < kLow; ++j) {
    lf_d[j] = 0; lf_bb[j] = 0; lf_si[j] = 0; lf_sstep[j] = 1; lf_fx[j] = -1;
    lf_al[j] = 1.0f; lf_hv[j] = 1.0f; lf_wl[j] = 0.5f;
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
    lf_bb[j] = bb - st;
    lf_si[j] = G::sl_off(d) + G::sl_idx(d, d == 0 ? -1 : l[0], d == 1 ? -1 : l[1], d == 2 ? -1 : l[2]);
    lf_sstep[j] = G::sl_step(d);
    lf_fx[j] = G::fx_off(d) + G::fx_idx(d, 0, l[0], l[1], l[2]);
    int gu[3] = {min(org[0] + l[0], a.n[0] - 1), min(org[1] + (DIM >= 2 ? l[1] : 0), a.n[1] - 1),
                 min(org[2] + (DIM >= 3 ? l[2] : 0), a.n[2] - 1)};
    int gl[3] = {gu[0], gu[1], gu[2]};
    const int od = d == 0 ? org[0] : d == 1 ? org[1] : org[2], nd = d == 0 ? a.n[0] : d == 1 ? a.n[1] : a.n[2];
    const int kl = d == 0 ? a.bc[0][0] : d == 1 ? a.bc[1][0] : a.bc[2][0];
    const int kh = d == 0 ? a.bc[0][1] : d == 1 ? a.bc[1][1] : a.bc[2][1];
    const int gud = min(od, nd - 1), gld = map_in(od - 1, nd, kl, kh);
    if (d == 0) { gu[0] = gud; gl[0] = gld; } else if (d == 1) { gu[1] = gud; gl[1] = gld; } else { gu[2] = gud; gl[2] = gld; }
    face_consts<float, VEL>(a, d, gl, gu, &lf_al[j], &lf_hv[j], &lf_wl[j]);
  }

  // ---- transport: Delta F_m of every angle quad ----------------------------------
  // One quad (two pairs: ka = 2j in the low halves, kb = 2j + 1 in the high
  // halves of every float4) per three barriers.  The own cell's values that a
  // later phase needs are read back from shared memory rather than held
  // across the barriers.
  //
  // A slot, extension item or low face whose index range the tile fills for
  // every thread is taken without a test (compile-time).  A tile with no
  // staged cell beyond a vacuum or inflow face and, with velocity, no face
  // of exactly zero velocity takes the loop without those two cases; the
  // choice is one per tile (a CTA-wide vote), so every warp runs the same
  // branch-free copy of the loop.
  float4 *O4 = reinterpret_cast<float4 *>(a.I_out);
  float4 pf[kSlots];   // quad j of each staged cell
#pragma unroll
  for (int s = 0; s < kSlots; ++s)
    pf[s] = slot_full(s) || sl_box[s] >= 0 ? I4[RT_IDX(sl_g[s], N)] : make_float4(0.f, 0.f, 0.f, 0.f);
  bool special = false;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) special |= sl_code[s] != 0;
  if (VEL) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) special |= iv_mean[d];
#pragma unroll
    for (int e = 0; e < kLow; ++e) special |= lf_fx[e] >= 0 && lf_wl[e] == 0.5f;
  }
  // The CTA-wide vote is also the barrier after which the shared table is
  // complete.  The warp vote on top of it changes no value (every lane
  // holds the same one; every tile shape is whole warps) but lets the
  // compiler see a warp-uniform choice, so the table loads of both copies
  // stay warp-uniform constant-bank loads.
  const bool general = __any_sync(0xffffffffu, __syncthreads_or(special) != 0);

  auto transport = [&](auto tag) {
    constexpr bool GEN = decltype(tag)::value;
    const float4 *qin = I4;
    float4 *qout = O4 + c;
    for (int j = 0; j < NQ; ++j) {
      const int m = 4 * j;   // angles past M read zero table entries
      // ---- phase 1: stage I~ and IV of the cross cells -----------------------
      {
        const float4 nx4 = tab4(j, 0), ny4 = tab4(j, 1), nz4 = tab4(j, 2);
        const f2 nxa = lo2(nx4), nya = lo2(ny4), nza = lo2(nz4);
        const f2 nxb = hi2(nx4), nyb = hi2(ny4), nzb = hi2(nz4);
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          if (!slot_full(s) && sl_box[s] < 0) continue;
          f2 Ia = lo2(pf[s]), Ib = hi2(pf[s]);
          if (GEN && sl_code[s]) {
            const int axis = (sl_code[s] >> 2) & 3, side = (sl_code[s] >> 4) & 1, face = axis * 2 + side;
            const float4 mu4 = tab4(j, axis);
            const f2 mua = lo2(mu4), mub = hi2(mu4);
            const bool infl = (sl_code[s] & 2) != 0;
            if (side ? (mua.x < 0.0f) : (mua.x > 0.0f)) Ia.x = infl ? inflow(face, m) : 0.0f;
            if (side ? (mua.y < 0.0f) : (mua.y > 0.0f)) Ia.y = infl ? inflow(face, m + 1) : 0.0f;
            if (side ? (mub.x < 0.0f) : (mub.x > 0.0f)) Ib.x = infl ? inflow(face, m + 2) : 0.0f;
            if (side ? (mub.y < 0.0f) : (mub.y > 0.0f)) Ib.y = infl ? inflow(face, m + 3) : 0.0f;
          }
          if (VEL) {
            const f2 w0 = dup(sl_w[s][0]), w1 = dup(sl_w[s][1]), w2 = dup(sl_w[s][2]);
            const f2 IVa = p_fma(nxa, w0, p_fma(nya, w1, p_mul(nza, w2)));
            const f2 IVb = p_fma(nxb, w0, p_fma(nyb, w1, p_mul(nzb, w2)));
            s_IV4[RT_IDX(sl_box[s], G::nbox)] = mk4(IVa, IVb);
            s_It4[RT_IDX(sl_box[s], G::nbox)] = mk4(p_fma(IVa, dup(-invC), Ia), p_fma(IVb, dup(-invC), Ib));
          } else {
            s_It4[RT_IDX(sl_box[s], G::nbox)] = mk4(Ia, Ib);
          }
        }
      }
      if (j + 1 < NQ) {
        qin += N;
#pragma unroll
        for (int s = 0; s < kSlots; ++s)
          if (slot_full(s) || sl_box[s] >= 0) pf[s] = qin[RT_IDX(sl_g[s], N)];
      }
      __syncthreads();

      // ---- phase 2: half slopes of I~ (own cell, extension cells) --------------
      {
        const float4 q0 = s_It4[RT_IDX(bo, G::nbox)];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const int st = bstride[d];
          const float4 qm = s_It4[RT_IDX(bo - st, G::nbox)], qp = s_It4[RT_IDX(bo + st, G::nbox)];
          s_sI4[RT_IDX(own_sl[d], G::SL3)] = mk4(vl_half2(lo2(qm), lo2(q0), lo2(qp)), vl_half2(hi2(qm), hi2(q0), hi2(qp)));
        }
#pragma unroll
        for (int e = 0; e < kExt; ++e) {
          if ((e + 1) * nthr > G::next && ext_si[e] < 0) continue;
          const int bb = ext_bb[e], st = ext_st[e];
          const float4 qm = s_It4[RT_IDX(bb - st, G::nbox)], qc = s_It4[RT_IDX(bb, G::nbox)],
                       qp = s_It4[RT_IDX(bb + st, G::nbox)];
          s_sI4[RT_IDX(ext_si[e], G::SL3)] = mk4(vl_half2(lo2(qm), lo2(qc), lo2(qp)), vl_half2(hi2(qm), hi2(qc), hi2(qp)));
        }
      }
      __syncthreads();

      // ---- phase 3: face fluxes (pre-multiplied by dt/dx) ----------------------
      float4 fhi[3];
      {
        const float4 q0 = s_It4[bo];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const int st = bstride[d];
          const int sl = own_sl[d], sn = own_sl[d] + G::sl_step(d);
          const float4 s0 = s_sI4[RT_IDX(sl, G::SL3)], q1 = s_It4[RT_IDX(bo + st, G::nbox)], s1 = s_sI4[RT_IDX(sn, G::SL3)];
          const float4 hc4 = tab4(j, 4 + d), hca4 = tab4(j, 7 + d), mud4 = tab4(j, 10 + d);
          f2 fa = face_flux2<false>(lo2(q0), lo2(s0), lo2(q1), lo2(s1), lo2(q0), lo2(q0), lo2(q0), lo2(q0),
                                    dup(fu_al[d]), dup(1.0f), dup(0.5f), lo2(hc4), lo2(hca4), lo2(mud4));
          f2 fb = face_flux2<false>(hi2(q0), hi2(s0), hi2(q1), hi2(s1), hi2(q0), hi2(q0), hi2(q0), hi2(q0),
                                    dup(fu_al[d]), dup(1.0f), dup(0.5f), hi2(hc4), hi2(hca4), hi2(mud4));
          if (VEL) {
            float4 iv;
            if (GEN && iv_mean[d]) {
              (void)RT_IDX(bo - st, G::nbox);
              (void)RT_IDX(bo + 2 * st, G::nbox);
              const float4 l = iv_state4(s_IV4, bo, st, fu_hv[d]), r = iv_state4(s_IV4, bo + st, st, -fu_hv[d]);
              iv = mk4(p_mul(dup(0.5f), p_add(lo2(l), lo2(r))), p_mul(dup(0.5f), p_add(hi2(l), hi2(r))));
            } else {
              (void)RT_IDX(bo + iv_off[d] - st, G::nbox);
              (void)RT_IDX(bo + iv_off[d] + st, G::nbox);
              iv = iv_state4(s_IV4, bo + iv_off[d], st, iv_sg[d]);
            }
            fa = p_fma(lo2(mud4), lo2(iv), fa);
            fb = p_fma(hi2(mud4), hi2(iv), fb);
          }
          fhi[d] = mk4(fa, fb);
          s_fx4[RT_IDX(own_fx[d] + G::fx_step(d), G::FX3)] = fhi[d];
        }
#pragma unroll
        for (int e = 0; e < kLow; ++e) {
          if ((e + 1) * nthr > G::nlow && lf_fx[e] < 0) continue;
          const int d = lf_d[e], bb = lf_bb[e], st = d == 0 ? 1 : bstride[d == 1 ? 1 : 2];
          const int si = lf_si[e], si1 = lf_si[e] + lf_sstep[e];
          const float4 qL = s_It4[RT_IDX(bb, G::nbox)], sL = s_sI4[RT_IDX(si, G::SL3)], qR = s_It4[RT_IDX(bb + st, G::nbox)],
                       sR = s_sI4[RT_IDX(si1, G::SL3)];
          const float4 hc4 = tab4(j, 4 + d), hca4 = tab4(j, 7 + d), mud4 = tab4(j, 10 + d);
          f2 fa = face_flux2<false>(lo2(qL), lo2(sL), lo2(qR), lo2(sR), lo2(qL), lo2(qL), lo2(qL), lo2(qL),
                                    dup(lf_al[e]), dup(1.0f), dup(0.5f), lo2(hc4), lo2(hca4), lo2(mud4));
          f2 fb = face_flux2<false>(hi2(qL), hi2(sL), hi2(qR), hi2(sR), hi2(qL), hi2(qL), hi2(qL), hi2(qL),
                                    dup(lf_al[e]), dup(1.0f), dup(0.5f), hi2(hc4), hi2(hca4), hi2(mud4));
          if (VEL) {
            // the low face lies between slots bb (below) and bb + st (above)
            const float wl = lf_wl[e], hv = lf_hv[e];
            float4 iv;
            if (GEN && wl == 0.5f) {
              (void)RT_IDX(bb - st, G::nbox);
              (void)RT_IDX(bb + 2 * st, G::nbox);
              const float4 l = iv_state4(s_IV4, bb, st, hv), r = iv_state4(s_IV4, bb + st, st, -hv);
              iv = mk4(p_mul(dup(0.5f), p_add(lo2(l), lo2(r))), p_mul(dup(0.5f), p_add(hi2(l), hi2(r))));
            } else {
              (void)RT_IDX((wl > 0.5f ? bb : bb + st) - st, G::nbox);
              (void)RT_IDX((wl > 0.5f ? bb : bb + st) + st, G::nbox);
              iv = iv_state4(s_IV4, wl > 0.5f ? bb : bb + st, st, wl > 0.5f ? hv : -hv);
            }
            fa = p_fma(lo2(mud4), lo2(iv), fa);
            fb = p_fma(hi2(mud4), hi2(iv), fb);
          }
          s_fx4[RT_IDX(lf_fx[e], G::FX3)] = mk4(fa, fb);
        }
      }
      __syncthreads();

      // ---- phase 4: Delta F of the quad ---------------------------------------
      {
        f2 da = dup(0.0f), db = dup(0.0f);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const float4 fl = s_fx4[RT_IDX(own_fx[d], G::FX3)];
          da = p_add(da, p_sub(lo2(fl), lo2(fhi[d])));
          db = p_add(db, p_sub(hi2(fl), hi2(fhi[d])));
        }
        if (valid) *qout = mk4(da, db);
      }
      qout += N;
    }
  };
  if (general)
    transport(BoolTag<true>{});
  else
    transport(BoolTag<false>{});

  if (!valid) return;

  // ---- per-cell constants of the implicit steps (see process_tile) -------------
  // Steps 4 and 5 are taken in deviations from the cell's center R (the
  // smallest I^n_m over its angles): every stored right-hand side, every
  // angle sum and both per-cell solves carry quantities of the size of I - R
  // rather than of I, and each per-cell solve is the exact sum of the
  // per-angle updates that follow it.  Float rounding then scales with the
  // spread of the intensities over angle (never above I_m itself, since R
  // <= I_m), and the energy the T^4 solve hands to the gas is the energy
  // the per-angle update takes from the radiation, step after step.
  float rho = a.rho[c], sa = a.sa[c], ss = a.ss[c], vt[3] = {0, 0, 0}, vin[3] = {0, 0, 0};
  const double T0 = a.T_in[c];
  // the cell's center: written by the step that produced I^n, or formed
  // here from I^n (padding angles excluded)
  float R;
  if (a.cen_in) {
    R = a.cen_in[c];
  } else {
    const float4 *p = I4 + c;
    R = p[0].x;
    for (int j = 0; j < NQ; ++j) {
      const float4 q = p[(long long)j * N];
      const int left = M - 4 * j;
      R = fminf(R, q.x);
      if (left > 1) R = fminf(R, q.y);
      if (left > 2) R = fminf(R, q.z);
      if (left > 3) R = fminf(R, q.w);
    }
  }
  if (VEL) {
    for (int d = 0; d < 3; ++d) vin[d] = a.v[d * N + c];
    if (a.estimate_v) {
      const float E = d2f_rn(a.mom_in[c]);
      const float h = 0.5f * dt * (sa + ss);
      for (int d = 0; d < 3; ++d) {
        const float Fd = d2f_rn(a.mom_in[(1 + d) * N + c]), Pdd = d2f_rn(a.mom_in[(4 + d) * N + c]);
        const float num = rho * vin[d] + h * (C * rho * vin[d] + a.P * Fd);
        const float den = rho + h * (C * rho + a.P * (E + Pdd) / C);
        vt[d] = num / den;
      }
    } else {
      vt[0] = vin[0]; vt[1] = vin[1]; vt[2] = vin[2];
    }
  }
  const bool to_scat = ss > sa;
  const float v2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
  const float A0 = 1.0f + dt * C * sa, A1 = dt * sa, kap = dt * sa / C;
  const float a0 = 1.0f + dt * C * ss, a1 = dt * ss;
  // beta_m = b_m + a1 C = 2 a1 vn - a1 (v.v + vn^2) / C (b_m of sec. 4.4)
  const float bt0 = -a1 * v2 * invC, bt1 = 2.0f * a1, bt2 = -a1 * invC;
  const float rd0 = VEL ? 0.0f : fast_rcp(A0);
  const float ra0 = VEL ? 0.0f : fast_rcp(a0);
  const f2 sc = dup(to_scat ? 1.0f : 0.0f), nsc = dup(to_scat ? 0.0f : 1.0f), Rv = dup(R);

  // ---- source loop: Q_m over Delta F, every angle sum of Steps 4 and 5 ---------
  // Per angle: d = A0 - A1 vn, a' = a0 - a1 vn (rd = 1/d, ra = 1/a'), rr = r_m
  // - R (Step 4's right-hand side: I^n, plus Delta F when it goes to Step 4),
  // stored Q_m = rd rr (+ Delta F when it goes to Step 5).  Sums: T_k = sum W
  // vn^k rd, U_k = sum W vn^k rd rr; with wa = W ra: As1 = sum wa, Va = sum wa
  // vn, Ad / Adv = sum wa rd (vn), AQ = sum wa Q; the beta-weighted Bs, Bv,
  // Bd, Bdv, BQ; pre = sum W n (I^n + Delta F - R).  The sums that depend on
  // the angle only through vn = n.v and its square (Vw = sum W vn, Gq = sum W
  // vn^2, Bw = sum beta W) are the table's own quadrature sums of W n and W n
  // n contracted with v, after the loop.
  f2 U0 = dup(0.0f), U1 = dup(0.0f), U2 = dup(0.0f);
  f2 T0p = dup(0.0f), T1p = dup(0.0f), T2p = dup(0.0f), T3p = dup(0.0f);
  f2 As1k = dup(0.0f), Vak = dup(0.0f), Adk = dup(0.0f), Advk = dup(0.0f), AQk = dup(0.0f);
  f2 Bsk = dup(0.0f), Bvk = dup(0.0f), Bdk = dup(0.0f), Bdvk = dup(0.0f), BQk = dup(0.0f);
  f2 pre0 = dup(0.0f), pre1 = dup(0.0f), pre2 = dup(0.0f);
  {
    const float4 *pi = I4 + c;
    float4 *pq = O4 + c;
    float4 i4n = *pi, d4n = *pq;   // the next quad's I^n and Delta F, loaded a quad ahead
#pragma unroll 2
    for (int j = 0; j < NQ; ++j) {
      const float4 i4 = i4n, d4 = d4n;
      if (j + 1 < NQ) {
        i4n = pi[N];
        d4n = pq[N];
      }
      f2 Qv[2];
      const float4 nx4 = tab4(j, 0), ny4 = tab4(j, 1), nz4 = tab4(j, 2), W4 = tab4(j, 3);
      const float4 wx4 = tab4(j, 13), wy4 = tab4(j, 14), wz4 = tab4(j, 15);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const f2 nx = h == 0 ? lo2(nx4) : hi2(nx4), ny = h == 0 ? lo2(ny4) : hi2(ny4);
        const f2 nz = h == 0 ? lo2(nz4) : hi2(nz4), Wm = h == 0 ? lo2(W4) : hi2(W4);
        const f2 I0 = h == 0 ? make_float2(i4.x, i4.y) : make_float2(i4.z, i4.w);
        const f2 dF = h == 0 ? make_float2(d4.x, d4.y) : make_float2(d4.z, d4.w);
        f2 vn = dup(0.0f), rd = dup(rd0), ra = dup(ra0);
        if (VEL) {
          vn = p_fma(nx, dup(vt[0]), p_fma(ny, dup(vt[1]), p_mul(nz, dup(vt[2]))));
          rd = p_rcp(p_fma(dup(-A1), vn, dup(A0)));
          ra = p_rcp(p_fma(dup(-a1), vn, dup(a0)));
        }
        const f2 g = p_sub(I0, Rv);
        const f2 gd = p_add(g, dF);   // I^n + Delta F - R
        const f2 rr = p_fma(nsc, dF, g);
        const f2 Q = p_fma(rd, rr, p_mul(sc, dF));
        Qv[h] = Q;
        // Every product below feeds a fused multiply-add as a factor, never
        // a separate add: the compiler may fuse a packed multiply into a
        // following add when the product has no other use, so a sum written
        // as add(mul) could round differently in the velocity and
        // no-velocity variants.  Written this way both round alike.
        const f2 wrd = p_mul(Wm, rd), wa = p_mul(Wm, ra);
        T0p = p_fma(Wm, rd, T0p);
        U0 = p_fma(wrd, rr, U0);
        if (VEL) {
          const f2 x1 = p_mul(wrd, vn), x2 = p_mul(x1, vn), y1 = p_mul(p_mul(wrd, rr), vn);
          T1p = p_fma(wrd, vn, T1p);
          T2p = p_fma(x1, vn, T2p);
          T3p = p_fma(x2, vn, T3p);
          U1 = p_add(U1, y1);
          U2 = p_fma(y1, vn, U2);
        }
        As1k = p_fma(Wm, ra, As1k);
        Adk = p_fma(wa, rd, Adk);
        AQk = p_fma(wa, Q, AQk);
        if (VEL) {
          const f2 war = p_mul(wa, rd);
          Vak = p_fma(wa, vn, Vak);
          Advk = p_fma(war, vn, Advk);
          const f2 bt = p_fma(vn, p_fma(dup(bt2), vn, dup(bt1)), dup(bt0));
          const f2 bwa = p_mul(bt, wa), bwar = p_mul(bwa, rd);
          Bsk = p_fma(bt, wa, Bsk);
          Bvk = p_fma(bwa, vn, Bvk);
          Bdk = p_fma(bwa, rd, Bdk);
          Bdvk = p_fma(bwar, vn, Bdvk);
          BQk = p_fma(bwa, Q, BQk);
        }
        pre0 = p_fma(h == 0 ? lo2(wx4) : hi2(wx4), gd, pre0);
        pre1 = p_fma(h == 0 ? lo2(wy4) : hi2(wy4), gd, pre1);
        pre2 = p_fma(h == 0 ? lo2(wz4) : hi2(wz4), gd, pre2);
      }
      *pq = make_float4(Qv[0].x, Qv[0].y, Qv[1].x, Qv[1].y);
      pi += N;
      pq += N;
    }
  }
  // Every sum is over the weights normalised to sum 1 (W / sum W, the float
  // table's sum being 1 + O(1e-8)): s (1 - wnorm) = s / sum W, formed as s -
  // s wnorm.  With sum W = 1 exact, isotropic equilibrium I_m = theta is a
  // fixed point of the energy row, as in the paper's quadrature.
  const float wn = a.wnorm;
  auto hsum = [wn](f2 x) {
    const float t = x.x + x.y;
    return fmaf(-t, wn, t);
  };
  const float T0s = hsum(T0p), T1s = hsum(T1p), T2s = hsum(T2p), T3s = hsum(T3p);
  const float U0s = hsum(U0), U1s = hsum(U1), U2s = hsum(U2);
  // sum W n_i and sum W n_i n_j (normalised, from the table in double)
  auto ms = [&](int i) { return a.msum[i][0] + a.msum[i][1]; };
  const float Vws = vt[0] * ms(1) + vt[1] * ms(2) + vt[2] * ms(3);
  const float Gqs = vt[0] * vt[0] * ms(4) + vt[1] * vt[1] * ms(5) + vt[2] * vt[2] * ms(6) +
                    2.0f * (vt[0] * vt[1] * ms(7) + vt[0] * vt[2] * ms(8) + vt[1] * vt[2] * ms(9));
  const float As1 = hsum(As1k), Va = hsum(Vak), Ad = hsum(Adk), Adv = hsum(Advk), AQ = hsum(AQk);
  const float Bs = hsum(Bsk), Bv = hsum(Bvk), Bd = hsum(Bdk), Bdv = hsum(Bdvk), BQ = hsum(BQk);
  const float Bw = bt0 + bt1 * Vws + bt2 * Gqs;

  // ---- Step 4 solve (sec. 4.3) in dth = theta - R ------------------------------
  // Each row reads I'_m - theta = rd (rr - dth - kappa S + 4 A1 theta vn), so
  // S = sum g I' (g = W (v.v + vn^2)), theta - J' and H' - S/C are affine in
  // dth, and the energy row is kv D + c0 + c1 dth(D) = 0 in D = T - T^n with
  // dth(D) = dth0 + ((T^n + D)^4 - (T^n)^4) / 4 pi.
  const float Gw = v2 + Gqs;
  const float G1 = v2 * T0s + T2s, Gr = v2 * U0s + U2s, Gv = v2 * T1s + T3s;
  const float den = 1.0f + kap * G1, Sg = Gw + 4.0f * A1 * Gv;
  const float S0 = (R * Sg + Gr) / den, S1 = (Sg - G1) / den;   // S = S0 + S1 dth
  const float q1 = -4.0f * A1 * T1s;
  const float Z0 = R * q1 + kap * S0 * T0s - U0s;               // theta - J' = Z0 + Z1 dth
  const float Z1 = q1 + T0s + kap * S1 * T0s;
  const float hv = Vws + 4.0f * A1 * T2s, ks = kap * T1s + invC;
  const float Y0 = R * hv + U1s - S0 * ks;                       // H' - S/C = Y0 + Y1 dth
  const float Y1 = hv - T1s - S1 * ks;
  const double kv = (double)rho * a.kv_per_rho;
  const double T0sq = T0 * T0;
  const float dth0 = (float)(T0sq * T0sq * (1.0 / (4.0 * kPi)) - (double)R);
  double T1 = T0;
  float dth = dth0;
  if (!a.hold_T) {
    const float beta = a.P * C * (1.0f - v2 * invC * invC) * sa;
    const float c0 = dt * (float(8.0 * kPi) * a.P * sa * Y0 + float(4.0 * kPi) * beta * Z0);
    const float c1 = dt * (float(8.0 * kPi) * a.P * sa * Y1 + float(4.0 * kPi) * beta * Z1);
    const float cc = c0 + c1 * dth0, c4 = c1 * float(1.0 / (4.0 * kPi));
    // Newton on D from 0; (T^n + D)^4 - (T^n)^4 = D (4 T^3 + D (6 T^2 + D (4 T
    // + D))) with T = T^n keeps every term of the row the size of D; the
    // stopping tolerance is the caller's (at least 1e-6 in float), then one
    // more step
    const float T0f = (float)T0, kvf = (float)kv;
    const float t2 = T0f * T0f, p3 = 4.0f * t2 * T0f, p2 = 6.0f * t2, p1 = 4.0f * T0f;
    const float rtol = fmaxf((float)a.newton_rtol, 1e-6f);
    const int max_it = a.newton_max_it;
    float d = 0.0f;
    int extra = -1, it;
    for (it = 0; it < max_it; ++it) {
      const float T = T0f + d;
      const float f = fmaf(kvf, d, fmaf(c4, d * fmaf(d, fmaf(d, p1 + d, p2), p3), cc));
      const float fp = fmaf(4.0f * c4, T * T * T, kvf);
      float dn = d - f / fp;
      if (!(T0f + dn > 0.0f)) dn = 0.5f * T - T0f;
      const float step = dn - d;
      d = dn;
      if (extra == 0) break;
      if (extra < 0 && fabsf(step) <= rtol * (T0f + d)) extra = 0;
    }
    T1 = T0 + (double)d;
    if (!(it < max_it && T1 > 0.0)) atomicAdd(a.status, 1);
    dth = dth0 + d * fmaf(d, fmaf(d, p1 + d, p2), p3) * float(1.0 / (4.0 * kPi));
  }
  const float th = R + dth;
  const float kS = kap * (S0 + S1 * dth);

  // ---- Step 5 solve (sec. 4.4) in sg = s1 + a1 C s2 and e2 = s2 - R ------------
  // Each row reads I''_m - s2 = ra (y_m + dth - e2 - sg + 4 a1 s2 vn) with
  // y_m = r'_m - theta = Q_m + rd (D0 + D1 vn); summing it against W (s2 =
  // sum W I'') and against beta W (sg = sum beta W I'') gives the 2x2 system.
  const float D0 = -(dth + kS), D1 = 4.0f * A1 * th;
  const float Ay = AQ + D0 * Ad + D1 * Adv, By = BQ + D0 * Bd + D1 * Bdv;
  const float fa = 4.0f * a1;
  const float m11 = 1.0f + Bs, m12 = Bs - Bw - fa * Bv, r1 = By + dth * Bs + R * (Bw + fa * Bv);
  const float m21 = As1, m22 = As1 - fa * Va, r2 = Ay + dth * As1 + fa * R * Va;
  const float det = m11 * m22 - m12 * m21;
  const float sg = (r1 * m22 - m12 * r2) / det;
  const float e2 = (m11 * r2 - m21 * r1) / det;
  const float E0c = dth - e2 - sg, E1c = fa * (R + e2);

  // ---- I^{n+1} over Q_m, quadrature (sec. 3) ---------------------------------
  // The moments are sums of the stored deviations I^{n+1} - R against W, W n
  // and W n n, plus R times the table's own sums of the same (mom_4pi_double).
  f2 mE = dup(0.0f), mF[3], mP[6];
  for (int i = 0; i < 3; ++i) mF[i] = dup(0.0f);
  for (int i = 0; i < 6; ++i) mP[i] = dup(0.0f);
  float cnext = __int_as_float(0x7f800000);   // the center of I^{n+1}: its smallest angle
  {
    float4 *pq = O4 + c;
    float4 q4 = *pq;
    for (int j = 0; j < NQ; ++j) {
      const float4 cur = q4;
      if (j + 1 < NQ) q4 = pq[N];   // the next quad, loaded before this one is overwritten
      f2 Iv[2];
      const float4 nx4 = tab4(j, 0), ny4 = tab4(j, 1), nz4 = tab4(j, 2), W4 = tab4(j, 3);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * j + h;
        const f2 nx = h == 0 ? lo2(nx4) : hi2(nx4), ny = h == 0 ? lo2(ny4) : hi2(ny4);
        const f2 nz = h == 0 ? lo2(nz4) : hi2(nz4), Wm = h == 0 ? lo2(W4) : hi2(W4);
        const f2 Q = h == 0 ? make_float2(cur.x, cur.y) : make_float2(cur.z, cur.w);
        f2 vn = dup(0.0f), rd = dup(rd0), ra = dup(ra0);
        if (VEL) {
          vn = p_fma(nx, dup(vt[0]), p_fma(ny, dup(vt[1]), p_mul(nz, dup(vt[2]))));
          rd = p_rcp(p_fma(dup(-A1), vn, dup(A0)));
          ra = p_rcp(p_fma(dup(-a1), vn, dup(a0)));
        }
        const f2 y = p_fma(rd, VEL ? p_fma(dup(D1), vn, dup(D0)) : dup(D0), Q);     // r'_m - theta
        const f2 z = p_add(y, VEL ? p_fma(dup(E1c), vn, dup(E0c)) : dup(E0c));
        f2 I1 = p_add(Rv, p_fma(ra, z, dup(e2)));                                  // R + (I'' - R)
        if (2 * k >= M) I1.x = 0.0f;          // padding angles stay zero
        else cnext = fminf(cnext, I1.x);
        if (2 * k + 1 >= M) I1.y = 0.0f;
        else cnext = fminf(cnext, I1.y);
        Iv[h] = I1;
        const f2 dv = p_sub(I1, Rv);   // the stored value's deviation (exact)
        const f2 wi = p_mul(Wm, dv);
        mE = p_fma(Wm, dv, mE);
        const f2 wx = p_mul(nx, wi), wy = p_mul(ny, wi), wz = p_mul(nz, wi);
        mF[0] = p_fma(nx, wi, mF[0]);
        mF[1] = p_fma(ny, wi, mF[1]);
        mF[2] = p_fma(nz, wi, mF[2]);
        mP[0] = p_fma(nx, wx, mP[0]);
        mP[1] = p_fma(ny, wy, mP[1]);
        mP[2] = p_fma(nz, wz, mP[2]);
        mP[3] = p_fma(ny, wx, mP[3]);
        mP[4] = p_fma(nz, wx, mP[4]);
        mP[5] = p_fma(nz, wy, mP[5]);
      }
      *pq = make_float4(Iv[0].x, Iv[0].y, Iv[1].x, Iv[1].y);
      pq += N;
    }
  }
  if (a.cen_out) a.cen_out[c] = cnext;
  a.mom_out[c] = mom_4pi_double(R, a.msum[0][0], a.msum[0][1], hsum(mE));
  float post[3];
  for (int i = 0; i < 3; ++i) {
    post[i] = hsum(mF[i]);
    a.mom_out[(1 + i) * N + c] = mom_4pi_double(R, a.msum[1 + i][0], a.msum[1 + i][1], post[i]);
  }
  for (int i = 0; i < 6; ++i)
    a.mom_out[(4 + i) * N + c] = mom_4pi_double(R, a.msum[4 + i][0], a.msum[4 + i][1], hsum(mP[i]));

  // ---- gas sources (sec. 4.3: Delta E_T, eqs. momentumchange, kinetichange)
  const float kmom = -float(4.0 * kPi) * a.P * invC;
  float dEK = 0.0f;
  const float pre[3] = {hsum(pre0), hsum(pre1), hsum(pre2)};
  for (int i = 0; i < 3; ++i) {
    const float dmom = kmom * (post[i] - pre[i]);
    a.dMom[i * N + c] = f2d_exact(dmom);
    const float m0 = rho * vin[i];
    dEK += ((m0 + dmom) * (m0 + dmom) - m0 * m0) / (2.0f * rho);
  }
  a.T_out[c] = T1;
  a.dEgas[c] = kv * (T1 - T0) + (double)dEK;
}

// Resident CTAs per SM a tile shape is compiled for: 512 threads per SM
// (128 registers per thread), so that smaller tiles run as several
// independent barrier domains per SM.
template <int NT>
constexpr int kQMinBlocks = NT >= 512 ? 1 : 512 / NT;

template <int DIM, bool VEL, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ, kQMinBlocks<TX * TY * TZ>)
    step_kernel_q(const StepArgs<float> a, const __grid_constant__ QTable<kQTabPairsSmall> qt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int o = a.outer_begin;
  process_tile_q<DIM, VEL, TX, TY, TZ, true, kQTabPairsSmall>(a, &qt, threadIdx.x, blockIdx.x + (DIM == 1 ? o : 0),
                                                              blockIdx.y + (DIM == 2 ? o : 0),
                                                              blockIdx.z + (DIM == 3 ? o : 0), smem_raw);
}

// Same kernel for angle sets beyond the launch-parameter table: the table is
// built in shared memory.
template <int DIM, bool VEL, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY * TZ, kQMinBlocks<TX * TY * TZ>) step_kernel_qs(const StepArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int o = a.outer_begin;
  process_tile_q<DIM, VEL, TX, TY, TZ, false, 2>(a, nullptr, threadIdx.x, blockIdx.x + (DIM == 1 ? o : 0),
                                                 blockIdx.y + (DIM == 2 ? o : 0), blockIdx.z + (DIM == 3 ? o : 0),
                                                 smem_raw);
}

// Host: the table of a launch (M <= 2 * kQTabPairsSmall).
inline void make_qtable(const StepArgs<float> &a, const float *host_ang, const float *host_inflow,
                        QTable<kQTabPairsSmall> *t) {
  fill_qtable(t, host_ang, a.M, a.C, a.dtdx, host_inflow);
}

template <int DIM, bool VEL, int TX, int TY, int TZ>
cudaError_t launch_shape_q(const StepArgs<float> &a, const QTable<kQTabPairsSmall> *qt, cudaStream_t s) {
  const bool param = qt != nullptr;
  const size_t sm = smem_bytes_q(DIM, a.M, VEL, TX, TY, TZ, param);
  dim3 block(TX * TY * TZ);
  dim3 grid((a.n[0] + TX - 1) / TX, (a.n[1] + TY - 1) / TY, (a.n[2] + TZ - 1) / TZ);
  if (a.outer_count > 0) (DIM == 3 ? grid.z : DIM == 2 ? grid.y : grid.x) = a.outer_count;
  if (param) {
    auto kern = step_kernel_q<DIM, VEL, TX, TY, TZ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, sm, s>>>(a, *qt);
  } else {
    auto kern = step_kernel_qs<DIM, VEL, TX, TY, TZ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, sm, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace stepk

}  // namespace rtg
