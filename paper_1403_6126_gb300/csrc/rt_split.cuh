// Two-kernel step for 3-D problems with float intensities (Jiang, Stone &
// Davis 2014, arXiv:1403.6126, secs. 3-4), the same arithmetic as the fused
// pair kernel (rt_step_pair.cuh), bitwise, split along the paper's own
// seams:
//
//   cell_kernel       per cell: the IV weights w = 3 J v of step n and, for
//                     every cell face, alpha (sec. 4.2) and the face velocity;
//   transport_kernel  Step 2 (sec. 4.2): Delta F_m of every cell and angle,
//                     written into the output intensity array;
//   source_kernel     Steps 3-5 and the quadrature: the implicit absorption
//                     and scattering of every cell over all its angles,
//                     I^{n+1}, E_r, F_r, P_r and the gas sources.
//
// transport_kernel gives each CTA a column of tx x ty cells and one angle
// pair and marches it along z.  The stencil along z lives in registers (each
// thread keeps I~ and IV of its own cell at z, z+1, z+2, its z slope and the
// flux through its lower z face), so shared memory holds one x-y layer with
// a two-cell x-y halo: per layer, one staged halo cell per ~1.6 cells
// instead of the ~2.75 of a 16x8x4 tile, and no staging along z at all.
// source_kernel is one thread per cell, no shared memory and no barriers;
// it reads I^n and Delta F, stores Q_m over Delta F and reads it back for
// the final pass, as the fused kernel does.
#pragma once

#include "rt_step_pair.cuh"

namespace rtg {

namespace split {

using stepk::dup;
using stepk::f2;
using stepk::face_flux2;
using stepk::KSum2;
using stepk::kHalo;
using stepk::kPi;
using stepk::map_in;
using stepk::p_add;
using stepk::p_fma;
using stepk::p_mul;
using stepk::p_rcp;
using stepk::p_sub;
using stepk::vl_half2;

// Per-cell scratch of cell_kernel: w[N] (w_x, w_y, w_z, 0) and face[6][N]
// (alpha, v_face) of the lower (rows 0-2) and upper (rows 3-5) face of each
// cell along x, y, z.
__host__ inline size_t scratch_bytes(long long N) { return (size_t)N * (sizeof(float4) + 6 * sizeof(float2)); }

template <bool VEL>
__global__ void __launch_bounds__(256) cell_kernel(const StepArgs<float> a) {
  const long long N = a.N;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % a.n[0]), y = (int)((c / a.n[0]) % a.n[1]), z = (int)(c / ((long long)a.n[0] * a.n[1]));
    float4 w = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (VEL) {
      const float w3 = float(3.0 / (4.0 * kPi)) * a.mom_in[c];
      w = make_float4(w3 * a.v[c], w3 * a.v[N + c], w3 * a.v[2 * N + c], 0.0f);
    }
    a.scr_w[c] = w;
    const int g[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
      for (int up = 0; up < 2; ++up) {
        int gl[3] = {g[0], g[1], g[2]}, gu[3] = {g[0], g[1], g[2]};
        if (up) gu[d] = map_in(g[d] + 1, a.n[d], a.bc[d][0], a.bc[d][1]);
        else gl[d] = map_in(g[d] - 1, a.n[d], a.bc[d][0], a.bc[d][1]);
        const long long cl = gl[0] + (long long)a.n[0] * (gl[1] + (long long)a.n[1] * gl[2]);
        const long long cu = gu[0] + (long long)a.n[0] * (gu[1] + (long long)a.n[1] * gu[2]);
        // as face_consts: alpha of a face is the mean of its cells'
        const float al = 0.5f * (stepk::alpha_of(a.dx[d], a.sa[cl] + a.ss[cl]) +
                                 stepk::alpha_of(a.dx[d], a.sa[cu] + a.ss[cu]));
        const float vf = VEL ? 0.5f * (a.v[d * N + cl] + a.v[d * N + cu]) : 0.0f;
        a.scr_face[(3 * up + d) * N + c] = make_float2(al, vf);
      }
    }
  }
}

// Boundary word of a position (grid coordinates, possibly outside) and the
// cell it reads: as the staging slots of process_tile2.
__device__ __forceinline__ int locate(const StepArgs<float> &a, int x, int y, int z, long long *g) {
  int p[3] = {x, y, z}, code = 0;
  for (int d = 0; d < 3; ++d) {
    if (p[d] < 0 || p[d] >= a.n[d]) {
      if (code == 0) code = 1 + 2 * d + (p[d] >= a.n[d] ? 1 : 0);
      p[d] = map_in(p[d], a.n[d], a.bc[d][0], a.bc[d][1]);
    }
  }
  if (code) {
    const int axis = (code - 1) >> 1, side = (code - 1) & 1;
    const int kind = a.bc[axis][side];
    code = (kind == stepk::BC_VACUUM || kind == stepk::BC_INFLOW)
               ? (1 | (kind == stepk::BC_INFLOW ? 2 : 0) | (axis << 2) | (side << 4))
               : 0;
  }
  *g = p[0] + (long long)a.n[0] * (p[1] + (long long)a.n[1] * p[2]);
  return code;
}

// Raw intensity pair and IV weights of a cell.
struct Raw {
  f2 I;
  float4 w;
};

template <bool VEL>
__device__ __forceinline__ Raw fetch(const StepArgs<float> &a, int m, bool second, long long g) {
  Raw r;
  r.I = make_float2(a.I_in[(long long)m * a.N + g], second ? a.I_in[(long long)(m + 1) * a.N + g] : 0.0f);
  r.w = VEL ? a.scr_w[g] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  return r;
}

// I~ and IV of a staged position for the angle pair (see process_tile2).
template <bool VEL>
__device__ __forceinline__ void value(const StepArgs<float> &a, const Raw &r, int code, int m, bool second, f2 nx, f2 ny,
                                      f2 nz, float invC, f2 *It, f2 *IV) {
  f2 I = r.I;
  if (code) {
    const int axis = (code >> 2) & 3, side = (code >> 4) & 1;
    const f2 mu = axis == 0 ? nx : axis == 1 ? ny : nz;
    const bool in0 = side ? (mu.x < 0.0f) : (mu.x > 0.0f);
    const bool in1 = second && (side ? (mu.y < 0.0f) : (mu.y > 0.0f));
    const float *row = a.inflow + (axis * 2 + side) * a.M + m;
    if (in0) I.x = (code & 2) ? row[0] : 0.0f;
    if (in1) I.y = (code & 2) ? row[1] : 0.0f;
  }
  if (VEL) {
    *IV = p_fma(nx, dup(r.w.x), p_fma(ny, dup(r.w.y), p_mul(nz, dup(r.w.z))));
    *It = p_fma(*IV, dup(-invC), I);
  } else {
    *IV = dup(0.0f);
    *It = I;
  }
}

// Shared-memory bytes of transport_kernel.
__host__ __device__ constexpr size_t transport_smem(int tx, int ty, bool vel) {
  return sizeof(f2) * (12 + (vel ? 2 : 1) * ((size_t)(tx + 4) * (ty + 4) + (size_t)(tx + 2) * ty + (size_t)tx * (ty + 2)) +
                       (size_t)(tx + 1) * ty + (size_t)tx * (ty + 1));
}

// Minimum resident CTAs per SM asked of the compiler for a transport tile.
__host__ __device__ constexpr int transport_min_blocks(int nt) { return nt >= 256 ? 3 : 6; }

template <bool VEL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, transport_min_blocks(TX * TY)) transport_kernel(const StepArgs<float> a) {
  constexpr int NT = TX * TY, BX = TX + 4, BY = TY + 4;
  constexpr int NHALO = 4 * TY + 4 * TX;        // x-y cross halo of one layer
  constexpr int KH = (NHALO + NT - 1) / NT;
  constexpr int NEXT = 2 * TY + 2 * TX;         // slope-extension items
  constexpr int NLOW = TY + TX;                 // lowest faces of the layer
  static_assert(NEXT <= NT && NLOW <= NT, "tile too narrow for one work item per thread");
  static_assert(KH <= 2, "halo needs at most two slots per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f2 *s_ang = reinterpret_cast<f2 *>(smem_raw);         // the pair: n (0-2), hc (3-5), hca (6-8), mud (9-11)
  f2 *s_It = s_ang + 12;                                // [BY][BX]
  f2 *s_IV = s_It + BX * BY;                            // [BY][BX]      (VEL)
  f2 *s_sxI = s_IV + (VEL ? BX * BY : 0);               // [TY][TX + 2]  x slopes, local x in [-1, TX]
  f2 *s_syI = s_sxI + (TX + 2) * TY;                    // [TY + 2][TX]  y slopes, local y in [-1, TY]
  f2 *s_sxV = s_syI + TX * (TY + 2);                    // (VEL)
  f2 *s_syV = s_sxV + (VEL ? (TX + 2) * TY : 0);        // (VEL)
  f2 *s_fx = s_syV + (VEL ? TX * (TY + 2) : 0);         // [TY][TX + 1]  x faces, face f between local f-1 and f
  f2 *s_fy = s_fx + (TX + 1) * TY;                      // [TY + 1][TX]

  const int M = a.M;
  const long long N = a.N, NXY = (long long)a.n[0] * a.n[1];
  const int m = 2 * blockIdx.x;
  const bool second = m + 1 < M;
  const int ntx = (a.n[0] + TX - 1) / TX, nty = (a.n[1] + TY - 1) / TY;
  const int tile = blockIdx.y + 65535 * blockIdx.z;   // x-y tiles beyond 65535 continue in blockIdx.z
  if (tile >= ntx * nty) return;                       // the whole CTA, before any barrier
  const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
  const int tid = threadIdx.x, lx = tid % TX, ly = tid / TX;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool valid = gx < a.n[0] && gy < a.n[1];
  const int gxc = min(gx, a.n[0] - 1), gyc = min(gy, a.n[1] - 1);
  const float invC = a.invC, C = a.C;

  // the angle pair (zeros for the weightless pad of an odd count), in shared
  // memory: the same for the whole CTA
  if (tid < 12) {
    const int d = tid % 3, kind = tid / 3;
    float v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int mm = m + h;
      float val = 0.0f;
      if (mm < M) {
        const float mu = a.ang[4 * mm + d], amu = mu < 0.0f ? -mu : mu;
        val = kind == 0   ? mu
              : kind == 1 ? 0.5f * C * mu * a.dtdx[d]
              : kind == 2 ? 0.5f * C * amu * a.dtdx[d]
                          : mu * a.dtdx[d];
      }
      v[h] = val;
    }
    s_ang[tid] = make_float2(v[0], v[1]);
  }
  __syncthreads();
  const f2 *nd = s_ang, *hc = s_ang + 3, *hca = s_ang + 6, *mud = s_ang + 9;

  // ---- per-thread work items, fixed along z ----------------------------------
  // halo slots: positions of the layer's cross halo (x halo rows, then y halo
  // columns); the cell index without z and the boundary word are fixed.
  int h_box[KH], h_code[KH];
  long long h_gxy[KH];
#pragma unroll
  for (int s = 0; s < KH; ++s) {
    h_box[s] = -1; h_code[s] = 0; h_gxy[s] = 0;
    const int k = tid + s * NT;
    if (k >= NHALO) continue;
    int bx, by;
    if (k < 4 * TY) {                 // x halo: layer h (0..3) of row r
      const int r = k % TY, h = k / TY;
      bx = h < 2 ? h : TX + h;        // 0, 1, TX+2, TX+3
      by = r + 2;
    } else {
      const int kk = k - 4 * TY, col = kk % TX, h = kk / TX;
      bx = col + 2;
      by = h < 2 ? h : TY + h;
    }
    h_box[s] = bx + BX * by;
    long long g;
    h_code[s] = locate(a, x0 + bx - 2, y0 + by - 2, 0, &g);   // z = 0 inside the grid: word from x, y
    h_gxy[s] = g;                                             // + z * NXY per layer
  }
  // slope-extension item: box position and stride of the stencil, target
  int e_bb = -1, e_st = 0, e_dst = 0;
  bool e_x = true;
  {
    const int e = tid;
    if (e < NEXT) {
      if (e < 2 * TY) {
        const int r = e % TY, right = e / TY;
        e_bb = (right ? TX + 2 : 1) + BX * (r + 2);
        e_st = 1;
        e_dst = (right ? TX + 1 : 0) + (TX + 2) * r;
        e_x = true;
      } else {
        const int ee = e - 2 * TY, col = ee % TX, top = ee / TX;
        e_bb = col + 2 + BX * (top ? TY + 2 : 1);
        e_st = BX;
        e_dst = col + TX * (top ? TY + 1 : 0);
        e_x = false;
      }
    }
  }
  // lowest-face item: the x face below local x = 0 of row r, or the y face
  // below local y = 0 of column c; its face data is the lower face of the
  // cell above it
  int l_bb = -1, l_dst = 0, l_si = 0, l_st = 1;
  bool l_x = true;
  long long l_cxy = 0;
  if (tid < NLOW) {
    if (tid < TY) {
      const int r = tid;
      l_x = true;
      l_bb = 1 + BX * (r + 2);
      l_st = 1;
      l_si = 0 + (TX + 2) * r;
      l_dst = 0 + (TX + 1) * r;
      l_cxy = min(x0, a.n[0] - 1) + (long long)a.n[0] * min(y0 + r, a.n[1] - 1);
    } else {
      const int col = tid - TY;
      l_x = false;
      l_bb = col + 2 + BX * 1;
      l_st = BX;
      l_si = col + TX * 0;
      l_dst = col + TX * 0;
      l_cxy = min(x0 + col, a.n[0] - 1) + (long long)a.n[0] * min(y0, a.n[1] - 1);
    }
  }
  const int bo = (lx + 2) + BX * (ly + 2);
  const long long own_xy = gxc + (long long)a.n[0] * gyc;
  const float dtdx0 = a.dtdx[0], dtdx1 = a.dtdx[1], dtdx2 = a.dtdx[2];
  auto hv_of = [](float vf, float dtdx) { return 1.0f - (vf < 0.0f ? -vf : vf) * dtdx; };
  auto wl_of = [](float vf) { return vf > 0.0f ? 1.0f : (vf < 0.0f ? 0.0f : 0.5f); };

  // ---- own column along z: prologue (z = -2 .. 2) ------------------------------
  f2 Pt[5], Pv[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    long long g;
    const int code = locate(a, gx, gy, j - 2, &g);
    const Raw r = fetch<VEL>(a, m, second, g);
    value<VEL>(a, r, code, m, second, nd[0], nd[1], nd[2], invC, &Pt[j], &Pv[j]);
  }
  f2 Q0t = Pt[2], Q0v = Pv[2], Q1t = Pt[3], Q1v = Pv[3], Q2t = Pt[4], Q2v = Pv[4];
  f2 SZt = vl_half2(Pt[1], Pt[2], Pt[3]), SZv = VEL ? vl_half2(Pv[1], Pv[2], Pv[3]) : dup(0.0f);
  f2 FZL;
  {
    const f2 smt = vl_half2(Pt[0], Pt[1], Pt[2]), smv = VEL ? vl_half2(Pv[0], Pv[1], Pv[2]) : dup(0.0f);
    const float2 fd = a.scr_face[2 * N + own_xy];            // lower z face of (x, y, 0)
    FZL = face_flux2<VEL>(Pt[1], smt, Pt[2], SZt, Pv[1], smv, Pv[2], SZv, dup(fd.x), dup(hv_of(fd.y, dtdx2)),
                          dup(wl_of(fd.y)), hc[2], hca[2], mud[2]);
  }

  // prefetch of layer 0's halo values and of the own cell at z = 3
  Raw h_raw[KH];
#pragma unroll
  for (int s = 0; s < KH; ++s)
    h_raw[s] = h_box[s] >= 0 ? fetch<VEL>(a, m, second, h_gxy[s]) : Raw{dup(0.0f), make_float4(0, 0, 0, 0)};
  // the own column's cell index without z and its boundary word from x, y;
  // positions beyond the z ends go through locate
  long long own_gxy;
  const int own_code_xy = locate(a, gx, gy, 0, &own_gxy);
  auto column = [&](int z, long long *g) {
    if (z >= 0 && z < a.n[2]) {
      *g = own_gxy + (long long)z * NXY;
      return own_code_xy;
    }
    return locate(a, gx, gy, z, g);
  };
  long long g3;
  int code3 = column(3, &g3);
  Raw r3 = fetch<VEL>(a, m, second, g3);

  const int nz = a.n[2];
  for (int z = 0; z < nz; ++z) {
    // ---- stage layer z: own cell from the column registers, the halo ----
    s_It[bo] = Q0t;
    if (VEL) s_IV[bo] = Q0v;
#pragma unroll
    for (int s = 0; s < KH; ++s) {
      if (h_box[s] < 0) continue;
      f2 t, v;
      value<VEL>(a, h_raw[s], h_code[s], m, second, nd[0], nd[1], nd[2], invC, &t, &v);
      s_It[h_box[s]] = t;
      if (VEL) s_IV[h_box[s]] = v;
    }
    // this layer's face data (used after two barriers), the next layer's
    // halo, and the own cell at z + 4
    const long long zoff = (long long)z * NXY;
    float2 cfu[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) cfu[d] = a.scr_face[(3 + d) * N + own_xy + zoff];
    const float2 cflo = l_bb >= 0 ? a.scr_face[(l_x ? 0 : 1) * N + l_cxy + zoff] : make_float2(1.0f, 0.0f);
    if (z + 1 < nz) {
      const long long off = zoff + NXY;
#pragma unroll
      for (int s = 0; s < KH; ++s)
        if (h_box[s] >= 0) h_raw[s] = fetch<VEL>(a, m, second, h_gxy[s] + off);
    }
    f2 n3t, n3v;
    value<VEL>(a, r3, code3, m, second, nd[0], nd[1], nd[2], invC, &n3t, &n3v);   // own cell at z + 3
    if (z + 1 < nz) {
      code3 = column(z + 4, &g3);
      r3 = fetch<VEL>(a, m, second, g3);
    }
    __syncthreads();

    // ---- half slopes: own x and y, extension cells, own z + 1 from registers ----
    const f2 sxt = vl_half2(s_It[bo - 1], Q0t, s_It[bo + 1]);
    const f2 syt = vl_half2(s_It[bo - BX], Q0t, s_It[bo + BX]);
    s_sxI[(lx + 1) + (TX + 2) * ly] = sxt;
    s_syI[lx + TX * (ly + 1)] = syt;
    f2 sxv = dup(0.0f), syv = dup(0.0f);
    if (VEL) {
      sxv = vl_half2(s_IV[bo - 1], Q0v, s_IV[bo + 1]);
      syv = vl_half2(s_IV[bo - BX], Q0v, s_IV[bo + BX]);
      s_sxV[(lx + 1) + (TX + 2) * ly] = sxv;
      s_syV[lx + TX * (ly + 1)] = syv;
    }
    if (e_bb >= 0) {
      const f2 st = vl_half2(s_It[e_bb - e_st], s_It[e_bb], s_It[e_bb + e_st]);
      (e_x ? s_sxI : s_syI)[e_dst] = st;
      if (VEL) (e_x ? s_sxV : s_syV)[e_dst] = vl_half2(s_IV[e_bb - e_st], s_IV[e_bb], s_IV[e_bb + e_st]);
    }
    const f2 SNt = vl_half2(Q0t, Q1t, Q2t), SNv = VEL ? vl_half2(Q0v, Q1v, Q2v) : dup(0.0f);
    __syncthreads();

    // ---- face fluxes: own upper x, y faces, the lowest faces, own upper z face ----
    const f2 fxh = face_flux2<VEL>(Q0t, sxt, s_It[bo + 1], s_sxI[(lx + 2) + (TX + 2) * ly], Q0v, sxv,
                                   VEL ? s_IV[bo + 1] : dup(0.0f), VEL ? s_sxV[(lx + 2) + (TX + 2) * ly] : dup(0.0f),
                                   dup(cfu[0].x), dup(hv_of(cfu[0].y, dtdx0)), dup(wl_of(cfu[0].y)), hc[0], hca[0],
                                   mud[0]);
    s_fx[(lx + 1) + (TX + 1) * ly] = fxh;
    const f2 fyh = face_flux2<VEL>(Q0t, syt, s_It[bo + BX], s_syI[lx + TX * (ly + 2)], Q0v, syv,
                                   VEL ? s_IV[bo + BX] : dup(0.0f), VEL ? s_syV[lx + TX * (ly + 2)] : dup(0.0f),
                                   dup(cfu[1].x), dup(hv_of(cfu[1].y, dtdx1)), dup(wl_of(cfu[1].y)), hc[1], hca[1],
                                   mud[1]);
    s_fy[lx + TX * (ly + 1)] = fyh;
    if (l_bb >= 0) {
      const f2 *sI = l_x ? s_sxI : s_syI;
      const f2 *sV = l_x ? s_sxV : s_syV;
      const int si1 = l_si + (l_x ? 1 : TX);
      const int d = l_x ? 0 : 1;
      const float dtdx = l_x ? dtdx0 : dtdx1;
      const f2 fl = face_flux2<VEL>(s_It[l_bb], sI[l_si], s_It[l_bb + l_st], sI[si1], VEL ? s_IV[l_bb] : dup(0.0f),
                                    VEL ? sV[l_si] : dup(0.0f), VEL ? s_IV[l_bb + l_st] : dup(0.0f),
                                    VEL ? sV[si1] : dup(0.0f), dup(cflo.x), dup(hv_of(cflo.y, dtdx)),
                                    dup(wl_of(cflo.y)), hc[d], hca[d], mud[d]);   // shared memory: no local array
      (l_x ? s_fx : s_fy)[l_dst] = fl;
    }
    const f2 fzh = face_flux2<VEL>(Q0t, SZt, Q1t, SNt, Q0v, SZv, Q1v, SNv, dup(cfu[2].x),
                                   dup(hv_of(cfu[2].y, dtdx2)), dup(wl_of(cfu[2].y)), hc[2], hca[2], mud[2]);
    __syncthreads();

    // ---- Delta F = sum over axes of (flux below - flux above) -------------
    f2 dF = dup(0.0f);
    dF = p_add(dF, p_sub(s_fx[lx + (TX + 1) * ly], fxh));
    dF = p_add(dF, p_sub(s_fy[lx + TX * ly], fyh));
    dF = p_add(dF, p_sub(FZL, fzh));
    if (valid) {
      const long long c = own_xy + (long long)z * NXY;
      a.I_out[(long long)m * N + c] = dF.x;
      if (second) a.I_out[(long long)(m + 1) * N + c] = dF.y;
    }
    // ---- advance the column --------------------------------------------------
    Q0t = Q1t; Q0v = Q1v;
    Q1t = Q2t; Q1v = Q2v;
    Q2t = n3t; Q2v = n3v;
    SZt = SNt; SZv = SNv;
    FZL = fzh;
  }
}

// Steps 3-5 and the quadrature of one cell over all angles; Delta F of the
// cell comes from transport_kernel in a.I_out.  Same arithmetic and order as
// the tail of process_tile2.
template <bool VEL>
__global__ void __launch_bounds__(256, 3) source_kernel(const StepArgs<float> a) {
  // pair table: n (0-2), W (3), W n (4-6), as process_tile2's table entries
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f2 *s_tab = reinterpret_cast<f2 *>(smem_raw);   // [K][8]
  const long long N = a.N;
  const int M = a.M, K = (M + 1) / 2;
  for (int i = threadIdx.x; i < 8 * K; i += blockDim.x) {
    const int k = i / 8, j = i % 8;
    float v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int mm = 2 * k + h;
      float val = 0.0f;
      if (mm < M && j < 7) val = j < 4 ? a.ang[4 * mm + j] : a.ang[4 * mm + 3] * a.ang[4 * mm + j - 4];
      v[h] = val;
    }
    s_tab[i] = make_float2(v[0], v[1]);
  }
  __syncthreads();
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;   // after the only barrier
  const float C = a.C, invC = a.invC, dt = a.dt;

  const float rho = a.rho[c], sa = a.sa[c], ss = a.ss[c];
  const double T0 = a.T_in[c];
  float vt[3] = {0, 0, 0}, vin[3] = {0, 0, 0};
  if (VEL) {
    for (int d = 0; d < 3; ++d) vin[d] = a.v[d * N + c];
    if (a.estimate_v) {
      const float E = a.mom_in[c];
      const float h = 0.5f * dt * (sa + ss);
      for (int d = 0; d < 3; ++d) {
        const float Fd = a.mom_in[(1 + d) * N + c], Pdd = a.mom_in[(4 + d) * N + c];
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
  const float bq0 = -dt * C * ss - dt * ss * v2 / C, bq1 = 2.0f * dt * ss, bq2 = -dt * ss / C;
  const float cq = -3.0f * dt * ss;
  const float apb0 = 1.0f - a1 * v2 * invC, apb2 = -a1 * invC;
  const float rd0 = VEL ? 0.0f : stepk::fast_rcp(A0);
  const float ra0 = VEL ? 0.0f : stepk::fast_rcp(a0);

  KSum2 U0, AQ;
  U0.zero();
  AQ.zero();
  f2 U1 = dup(0.0f), U2 = dup(0.0f), BQ = dup(0.0f), pre0 = dup(0.0f), pre1 = dup(0.0f), pre2 = dup(0.0f);
  f2 T0p = dup(0.0f), T1p = dup(0.0f), T2p = dup(0.0f), T3p = dup(0.0f);
  f2 Apk = dup(0.0f), Adk = dup(0.0f), As1k = dup(0.0f), Acck = dup(0.0f);
  f2 Bpk = dup(0.0f), Bdk = dup(0.0f), Bcck = dup(0.0f), B1pk = dup(0.0f);
  float *out = a.I_out + c;
  const float *in = a.I_in + c;

  auto angle = [&](int k, f2 *nx, f2 *ny, f2 *nz, f2 *W, f2 *Wn) {
    const f2 *t = s_tab + 8 * k;
    *nx = t[0];
    *ny = t[1];
    *nz = t[2];
    *W = t[3];
    Wn[0] = t[4];
    Wn[1] = t[5];
    Wn[2] = t[6];
  };

  for (int k = 0; k < K; ++k) {
    const int m = 2 * k;
    const bool second = m + 1 < M;
    f2 nx, ny, nz, Wm, Wn[3];
    angle(k, &nx, &ny, &nz, &Wm, Wn);
    const f2 I0 = make_float2(in[(long long)m * N], second ? in[(long long)(m + 1) * N] : 0.0f);
    const f2 dF = make_float2(out[(long long)m * N], second ? out[(long long)(m + 1) * N] : 0.0f);
    const f2 full = p_add(I0, dF);
    f2 vn = dup(0.0f), rd = dup(rd0), ra = dup(ra0);
    if (VEL) {
      vn = p_fma(nx, dup(vt[0]), p_fma(ny, dup(vt[1]), p_mul(nz, dup(vt[2]))));
      rd = p_rcp(p_fma(dup(-A1), vn, dup(A0)));
      ra = p_rcp(p_fma(dup(-a1), vn, dup(a0)));
    }
    const f2 qa = p_mul(to_scat ? I0 : full, rd);
    const f2 Q = to_scat ? p_add(qa, dF) : qa;
    out[(long long)m * N] = Q.x;
    if (second) out[(long long)(m + 1) * N] = Q.y;
    // intensity-dependent sums (as the transport loop of process_tile2)
    const f2 wq = p_mul(Wm, qa);
    U0.part = p_add(U0.part, wq);
    if (VEL) {
      const f2 y1 = p_mul(wq, vn);
      U1 = p_add(U1, y1);
      U2 = p_fma(y1, vn, U2);
    }
    const f2 wa = p_mul(Wm, ra);
    AQ.part = p_fma(wa, Q, AQ.part);
    const f2 bm = VEL ? p_fma(vn, p_fma(dup(bq2), vn, dup(bq1)), dup(bq0)) : dup(bq0);
    BQ = p_fma(p_mul(bm, wa), Q, BQ);
    pre0 = p_fma(Wn[0], full, pre0);
    pre1 = p_fma(Wn[1], full, pre1);
    pre2 = p_fma(Wn[2], full, pre2);
    if ((k & 3) == 3) { U0.fold(); AQ.fold(); }
  }
  // velocity-only sums (as the second loop of process_tile2)
  for (int k = 0; k < K; ++k) {
    f2 nx, ny, nz, Wm, Wn[3];
    angle(k, &nx, &ny, &nz, &Wm, Wn);
    f2 vn = dup(0.0f), rd = dup(rd0), ra = dup(ra0);
    if (VEL) {
      vn = p_fma(nx, dup(vt[0]), p_fma(ny, dup(vt[1]), p_mul(nz, dup(vt[2]))));
      rd = p_rcp(p_fma(dup(-A1), vn, dup(A0)));
      ra = p_rcp(p_fma(dup(-a1), vn, dup(a0)));
    }
    const f2 wrd = p_mul(Wm, rd);
    T0p = p_add(T0p, wrd);
    if (VEL) {
      const f2 x1 = p_mul(wrd, vn), x2 = p_mul(x1, vn);
      T1p = p_add(T1p, x1);
      T2p = p_add(T2p, x2);
      T3p = p_fma(x2, vn, T3p);
    }
    const f2 pe = p_mul(dup(A1), p_mul(p_fma(dup(3.0f), vn, dup(C)), rd));
    const f2 wa = p_mul(Wm, ra);
    Apk = p_fma(wa, pe, Apk);
    Adk = p_fma(wa, rd, Adk);
    As1k = p_add(As1k, wa);
    if (VEL) {
      const f2 bm = p_fma(vn, p_fma(dup(bq2), vn, dup(bq1)), dup(bq0));
      const f2 cm = p_mul(dup(cq), vn);
      const f2 bwa = p_mul(bm, wa);
      Acck = p_fma(cm, wa, Acck);
      Bpk = p_fma(bwa, pe, Bpk);
      Bdk = p_fma(bwa, rd, Bdk);
      Bcck = p_fma(cm, bwa, Bcck);
      B1pk = p_fma(wa, p_fma(vn, p_fma(dup(apb2), vn, dup(a1)), dup(apb0)), B1pk);
    } else {
      const f2 bwa = p_mul(dup(bq0), wa);
      Bpk = p_fma(bwa, pe, Bpk);
      Bdk = p_fma(bwa, rd, Bdk);
      B1pk = p_add(B1pk, wa);
    }
  }
  const float T0s = T0p.x + T0p.y, T1s = T1p.x + T1p.y, T2s = T2p.x + T2p.y, T3s = T3p.x + T3p.y;
  const float Ap = Apk.x + Apk.y, Ad = Adk.x + Adk.y, As1 = As1k.x + As1k.y, Acc = Acck.x + Acck.y;
  const float Bp = Bpk.x + Bpk.y, Bd = Bdk.x + Bdk.y, Bcc = Bcck.x + Bcck.y, B1p = B1pk.x + B1pk.y;

  // ---- Step 4 solve (see process_tile2) -------------------------------------
  const float Wr = U0.total(), Vr = U1.x + U1.y, Gr = v2 * Wr + (U2.x + U2.y);
  const float W1 = T0s, V1 = T1s, G1 = v2 * T0s + T2s;
  const float Ve = A1 * (C * T1s + 3.0f * T2s);
  const float Ge = A1 * (C * (v2 * T0s + T2s) + 3.0f * (v2 * T1s + T3s));
  const float Wq = T0s - 4.0f * A1 * T1s;
  const float den = 1.0f + kap * G1;
  const float S0 = Gr / den, S1 = Ge / den;
  const float J0 = Wr - kap * S0 * W1;
  const float H0 = Vr - kap * S0 * V1, H1 = Ve - kap * S1 * V1;
  const float omJ1 = Wq + kap * S1 * W1;
  const double kv = (double)rho * a.kv_per_rho;
  double T1 = T0;
  if (!a.hold_T) {
    const float beta = a.P * C * (1.0f - v2 * invC * invC) * sa;
    const float c0r = dt * (float(8.0 * kPi) * a.P * sa * (H0 - S0 * invC) - float(4.0 * kPi) * beta * J0);
    const float c4 = dt * (2.0f * a.P * sa * (H1 - S1 * invC) + beta * omJ1);
    const float T0f = (float)T0, kvf = (float)kv;
    float d = 0.0f;
    int extra = -1, it;
    for (it = 0; it < 40; ++it) {
      const float T = T0f + d, T2 = T * T;
      const float f = c4 * T2 * T2 + kvf * d + c0r;
      const float fp = 4.0f * c4 * T2 * T + kvf;
      float dn = d - f / fp;
      if (!(T0f + dn > 0.0f)) dn = 0.5f * T - T0f;
      const float step = dn - d;
      d = dn;
      if (extra == 0) break;
      if (extra < 0 && fabsf(step) <= 2e-7f * (T0f + d)) extra = 0;
    }
    double dd = (double)d;
    const double T = T0 + dd, T2 = T * T;
    const double f = (double)c4 * T2 * T2 + kv * dd + (double)c0r;
    const float fp = 4.0f * c4 * (float)(T2 * T) + kvf;
    dd -= f * (double)(1.0f / fp);
    if (!(it < 40 && (T0 + dd) > 0.0)) atomicAdd(a.status, 1);
    T1 = T0 + dd;
  }
  const float T1r = (float)T1, T1sq = T1r * T1r;
  const float th = T1sq * T1sq * float(1.0 / (4.0 * kPi));
  const float S = S0 + th * S1;
  const float kS = kap * S;

  // ---- Step 5 solve --------------------------------------------------------------
  const float Ar = AQ.total() + th * Ap - kS * Ad;
  const float Br = (BQ.x + BQ.y) + th * Bp - kS * Bd;
  const float m11 = B1p, m12 = Bcc, m21 = As1, m22 = 1.0f + Acc;
  const float det = m11 * m22 - m12 * m21;
  const float s1 = (Br * m22 - m12 * Ar) / det;
  const float s2 = (m11 * Ar - m21 * Br) / det;

  // ---- I^{n+1} over Q_m, quadrature (sec. 3) ---------------------------------------
  KSum2 mE, mF[3], mP[6];
  mE.zero();
  for (int i = 0; i < 3; ++i) mF[i].zero();
  for (int i = 0; i < 6; ++i) mP[i].zero();
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    const int m = 2 * k;
    const bool second = m + 1 < M;
    f2 nx, ny, nz, Wm, Wn[3];
    angle(k, &nx, &ny, &nz, &Wm, Wn);
    const f2 Q = make_float2(out[(long long)m * N], second ? out[(long long)(m + 1) * N] : 0.0f);
    f2 vn = dup(0.0f), rd = dup(rd0), ra = dup(ra0);
    if (VEL) {
      vn = p_fma(nx, dup(vt[0]), p_fma(ny, dup(vt[1]), p_mul(nz, dup(vt[2]))));
      rd = p_rcp(p_fma(dup(-A1), vn, dup(A0)));
      ra = p_rcp(p_fma(dup(-a1), vn, dup(a0)));
    }
    const f2 pe = p_mul(dup(A1), p_mul(p_fma(dup(3.0f), vn, dup(C)), rd));
    const f2 rs = p_fma(pe, dup(th), p_fma(rd, dup(-kS), Q));
    const f2 cm = p_mul(dup(cq), vn);
    const f2 I1 = p_mul(p_fma(cm, dup(-s2), p_sub(rs, dup(s1))), ra);
    out[(long long)m * N] = I1.x;
    if (second) out[(long long)(m + 1) * N] = I1.y;
    const f2 wi = p_mul(Wm, I1);
    mE.part = p_add(mE.part, wi);
    const f2 wx = p_mul(nx, wi), wy = p_mul(ny, wi), wz = p_mul(nz, wi);
    mF[0].part = p_add(mF[0].part, wx);
    mF[1].part = p_add(mF[1].part, wy);
    mF[2].part = p_add(mF[2].part, wz);
    mP[0].part = p_fma(nx, wx, mP[0].part);
    mP[1].part = p_fma(ny, wy, mP[1].part);
    mP[2].part = p_fma(nz, wz, mP[2].part);
    mP[3].part = p_fma(ny, wx, mP[3].part);
    mP[4].part = p_fma(nz, wx, mP[4].part);
    mP[5].part = p_fma(nz, wy, mP[5].part);
    if ((k & 3) == 3) {
      mE.fold();
      for (int i = 0; i < 3; ++i) mF[i].fold();
      for (int i = 0; i < 6; ++i) mP[i].fold();
    }
  }
  const float fourpi = float(4.0 * kPi);
  a.mom_out[c] = fourpi * mE.total();
  float post[3];
  for (int i = 0; i < 3; ++i) {
    post[i] = mF[i].total();
    a.mom_out[(1 + i) * N + c] = fourpi * post[i];
  }
  for (int i = 0; i < 6; ++i) a.mom_out[(4 + i) * N + c] = fourpi * mP[i].total();
  const float kmom = -fourpi * a.P * invC;
  float dEK = 0.0f;
  const float pre[3] = {pre0.x + pre0.y, pre1.x + pre1.y, pre2.x + pre2.y};
  for (int i = 0; i < 3; ++i) {
    const float dmom = kmom * (post[i] - pre[i]);
    a.dMom[i * N + c] = dmom;
    const float m0 = rho * vin[i];
    dEK += ((m0 + dmom) * (m0 + dmom) - m0 * m0) / (2.0f * rho);
  }
  a.T_out[c] = T1;
  a.dEgas[c] = kv * (T1 - T0) + (double)dEK;
}

// The three launches of one step; TX x TY is the transport kernel's column
// tile.  a.scr_w / a.scr_face must hold scratch_bytes(N).
template <bool VEL, int TX, int TY>
cudaError_t launch(const StepArgs<float> &a, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long cells_blocks = (a.N + 255) / 256;
  cell_kernel<VEL><<<(int)std::min<long long>(cells_blocks, 8LL * sms), 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t sm = transport_smem(TX, TY, VEL);
  auto tk = transport_kernel<VEL, TX, TY>;
  if ((e = cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess) return e;
  const int ntx = (a.n[0] + TX - 1) / TX, nty = (a.n[1] + TY - 1) / TY, nt = ntx * nty;
  tk<<<dim3((a.M + 1) / 2, std::min(nt, 65535), (nt + 65534) / 65535), TX * TY, sm, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  source_kernel<VEL><<<(unsigned)cells_blocks, 256, sizeof(f2) * 8 * ((a.M + 1) / 2), s>>>(a);
  return cudaGetLastError();
}

}  // namespace split

}  // namespace rtg
