// Assembly kernels: the EFIE blocks T_A and V (Sec. 2), the plane-wave
// excitation e and the radiation vector for the far field.
//
// Every cell pair (s, t) is reduced to four moments in centroid-local
// coordinates rho = r - c_s, rho' = r' - c_t:
//   I0 = int int G,  Ir = int int rho G,  Irp = int int rho' G,  Irr = int int rho.rho' G,
// G = e^{ikR} / (4 pi R).  The local RWG half-function of cell s opposite its
// vertex i is sigma (r - P_i) / (2 A_s) (Eq. RWGdef), so the pair contributes
//   sigma_i sigma_j [Irr - b_j.Ir - a_i.Irp + (a_i.b_j) I0] / (4 A_s A_t)
// to [T_A]_{m_i n_j} (a_i = P_i - c_s, b_j = P_j - c_t), and I0 / (A_s A_t)
// to V_st (p = 1/A, Eq. patchstddef).
//
// Far pairs (no shared vertex): 7 x 7 product of the 7-point rule, FP32,
// one unordered pair per thread, both (s,t) and (t,s) written.
// Near pairs (a shared vertex): FP64, G split as 1/(4 pi R) + (e^{ikR}-1)/(4 pi R);
// the first term integrated over the source cell in closed form (integrals of
// 1/R and (r'-p)/R over a flat triangle by Stokes' theorem, Wilton et al. 1984),
// the second by the 7-point rule; the result is the mean of both orders.
#include <cuda_runtime.h>

#include <cmath>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

constexpr int TILE = 32;          // cells per tile side
constexpr int FAR_THREADS = 256;  // 32 s-cells x 8 t-lanes
constexpr float INV_4PI_F = 0.0795774715459476679f;
constexpr double INV_4PI = 0.0795774715459476679;

// 1/sqrt(x) with subnormal inputs and results flushed to zero: the hardware approximation alone,
// without the rescaling a subnormal operand would need (far-pair distances are far from it)
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// sin and cos of |r| <= pi/4 in FP32: Taylor series of sin to r^9 and of cos to r^8
// (truncation below 4e-9).
__device__ __forceinline__ void sincos_quarter(float r, float* s, float* c) {
  const float r2 = r * r;
  // sin r = r (1 - r^2/6 + r^4/120 - r^6/5040 + r^8/362880)
  float ps = fmaf(r2, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = fmaf(r2, ps, 1.0f / 120.0f);
  ps = fmaf(r2, ps, -1.0f / 6.0f);
  *s = fmaf(r * r2, ps, r);
  // cos r = 1 - r^2/2 + r^4/24 - r^6/720 + r^8/40320
  float pc = fmaf(r2, 1.0f / 40320.0f, -1.0f / 720.0f);
  pc = fmaf(r2, pc, 1.0f / 24.0f);
  pc = fmaf(r2, pc, -0.5f);
  *c = fmaf(r2, pc, 1.0f);
}

// sin and cos of |r| <= 1/20 in FP32: sin to r^3 (truncation r^4/120 <= 6e-8 relative, the FP32
// rounding) and cos to r^4 (below 3e-11)
__device__ __forceinline__ void sincos_twentieth(float r, float* s, float* c) {
  const float r2 = r * r;
  *s = fmaf(r * r2, -1.0f / 6.0f, r);
  *c = fmaf(r2, fmaf(r2, 1.0f / 24.0f, -0.5f), 1.0f);
}

// sin and cos of x >= 0 in FP32.  Cody and Waite's reduction (1980): q = nearest integer to
// x 2/pi, r = x - q pi/2 with pi/2 split into a short leading part (q times it is exact for
// q < 2^16) and a remainder; then the series above on |r| <= pi/4 and the quadrant of q.
__device__ __forceinline__ void sincos_far(float x, float* s, float* c) {
  constexpr float TWO_OVER_PI = 0.636619772367581343f;
  constexpr float PIO2_HI = 1.5703125f;                    // 8 significant bits
  constexpr float PIO2_LO = 4.83826794896619231e-4f;       // pi/2 - PIO2_HI
  const float q = rintf(x * TWO_OVER_PI);
  const float r = fmaf(-q, PIO2_LO, fmaf(-q, PIO2_HI, x));
  float sr, cr;
  sincos_quarter(r, &sr, &cr);
  const int quad = ((int)q) & 3;  // x = q pi/2 + r
  const float ss = (quad & 1) ? cr : sr, cc = (quad & 1) ? sr : cr;
  *s = (quad & 2) ? -ss : ss;
  *c = ((quad + 1) & 2) ? -cc : cc;
}

__device__ __forceinline__ void atomic_add_c64(float2* p, float re, float im) {
  atomicAdd(p, make_float2(re, im));
}

// shared-memory image of one tile of cells
struct TileCells {
  float rho[TILE][21];
  float wq[TILE][7];    // weight x area
  float cen_hi[TILE][3];
  float cen_lo[TILE][3];
  float aloc[TILE][9];
  float inv_area[TILE];
  float rq[TILE];       // largest distance of a quadrature point from the centroid
  int32_t vid[TILE][3];
  int32_t edge[TILE][3];
  float sign[TILE][3];
};

// Source-side quadrature data of the t tile as the evaluation loop reads it: per cell and point j
// (-2 rho'_j, |rho'_j|^2) in one 16-byte word, and the weight x area / (4 pi).  A warp reads eight
// cells at once; row strides of 28 and 7 words put them on distinct banks.
struct SourceTile {
  float4 qn[TILE][7];
  float w[TILE][7];
};

// Both tiles of a block and the source data, loaded by all threads: first coalesced copies of the
// per-cell arrays (cells past the end read cell 0 and get vertex ids that match nothing), then the
// derived quantities.  Ends with the block synchronised.
__device__ void load_tiles(TileCells& S, TileCells& T, SourceTile& Q, const DeviceGeometry& g, int bs, int bt) {
  const int nt = blockDim.x;
  for (int side = 0; side < 2; ++side) {
    TileCells& X = side ? T : S;
    const int base = side ? bt : bs;
    auto cell = [&](int q) { return base + q < g.nc ? base + q : 0; };
    for (int it = threadIdx.x; it < TILE * 21; it += nt) X.rho[it / 21][it % 21] = g.rho[21 * cell(it / 21) + it % 21];
    for (int it = threadIdx.x; it < TILE * 9; it += nt) X.aloc[it / 9][it % 9] = g.aloc[9 * cell(it / 9) + it % 9];
    for (int it = threadIdx.x; it < TILE * 7; it += nt) X.wq[it / 7][it % 7] = g.wq[7 * cell(it / 7) + it % 7];
    for (int it = threadIdx.x; it < TILE * 3; it += nt) {
      const int q = it / 3, e = it % 3, c = cell(q);
      X.cen_hi[q][e] = g.cen_hi[3 * c + e];
      X.cen_lo[q][e] = g.cen_lo[3 * c + e];
      X.vid[q][e] = base + q < g.nc ? g.tris[3 * c + e] : -1 - q;
      X.edge[q][e] = g.cell_edges[3 * c + e];
      X.sign[q][e] = (float)g.cell_sign[3 * c + e];
    }
    for (int q = threadIdx.x; q < TILE; q += nt) X.inv_area[q] = g.inv_area[cell(q)];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < 2 * TILE; it += nt) {
    TileCells& X = it < TILE ? S : T;
    const int q = it % TILE;
    float rq2 = 0.f;
    for (int j = 0; j < 7; ++j) {
      const float a = X.rho[q][3 * j], b = X.rho[q][3 * j + 1], c = X.rho[q][3 * j + 2];
      rq2 = fmaxf(rq2, fmaf(a, a, fmaf(b, b, c * c)));
    }
    X.rq[q] = sqrtf(rq2) * 1.0001f;  // rounding margin
  }
  for (int it = threadIdx.x; it < TILE * 7; it += nt) {
    const int q = it / 7, j = it % 7;
    const float x = T.rho[q][3 * j], y = T.rho[q][3 * j + 1], z = T.rho[q][3 * j + 2];
    Q.qn[q][j] = make_float4(-2.f * x, -2.f * y, -2.f * z, fmaf(x, x, fmaf(y, y, z * z)));
    Q.w[q][j] = T.wq[q][j] * INV_4PI_F;
  }
  __syncthreads();
}

// the four moments of a far pair (Sec. 2; I0, Ir, Irp, Irr with G = e^{ik(R - phase0/k)} / (4 pi R))
struct FarMoments {
  float I0r = 0.f, I0i = 0.f, Irr_r = 0.f, Irr_i = 0.f;
  float Ir_r[3] = {0.f, 0.f, 0.f}, Ir_i[3] = {0.f, 0.f, 0.f};
  float Ip_r[3] = {0.f, 0.f, 0.f}, Ip_i[3] = {0.f, 0.f, 0.f};
  // multiply every moment by e^{i phi}
  __device__ __forceinline__ void rotate(float phi) {
    float sn, cs;
    sincos_far(phi, &sn, &cs);
    auto rot = [&](float& re, float& im) {
      const float a = re, b = im;
      re = fmaf(a, cs, -b * sn);
      im = fmaf(a, sn, b * cs);
    };
    rot(I0r, I0i);
    rot(Irr_r, Irr_i);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      rot(Ir_r[e], Ir_i[e]);
      rot(Ip_r[e], Ip_i[e]);
    }
  }
};

// 7 x 7 product rule over the pair (s outer, t source).  For outer point i, D = c_s + rho_i - c_t
// and R^2 = |D|^2 + |rho'_j|^2 + D.(-2 rho'_j): four operations per evaluation for R^2, the
// source data read from shared memory where they are used.  SHIFTED > 0: the phase of each
// evaluation is k R - k Rc with |k R - k Rc| <= pi/4 (SHIFTED 1, series to r^9 / r^8) or <= 1/20
// (SHIFTED 2: sin to r^3, cos to r^2, truncation below 3e-7) or <= 3.4e-4 (SHIFTED 3: sin x = x,
// cos x = 1), no range reduction; 0: sin and cos of k R with the reduction (k R < 1.029e5, which
// the host checks at op creation).  The rho' moments come out of the loop against -2 rho' and are
// scaled back at the end.
template <int SHIFTED, int UNROLL>
__device__ __forceinline__ void far_moments(const TileCells& S, int sl, const SourceTile& Q, int tl, const float (&d)[3],
                                            float k, float kref, FarMoments& M) {
#pragma unroll 1
  for (int i = 0; i < 7; ++i) {
    const float rsx = S.rho[sl][3 * i], rsy = S.rho[sl][3 * i + 1], rsz = S.rho[sl][3 * i + 2], wsi = S.wq[sl][i];
    const float Dx = d[0] + rsx, Dy = d[1] + rsy, Dz = d[2] + rsz;
    const float A = fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz));
    float s0r = 0.f, s0i = 0.f;
    float s1r[3] = {0.f, 0.f, 0.f}, s1i[3] = {0.f, 0.f, 0.f};
#pragma unroll UNROLL
    for (int j = 0; j < 7; ++j) {
      const float4 q = Q.qn[tl][j];
      const float r2 = fmaf(Dx, q.x, fmaf(Dy, q.y, fmaf(Dz, q.z, A + q.w)));
      const float rinv = rsqrt_ftz(r2);
      const float R = r2 * rinv;
      float sn, cs;
      if (SHIFTED == 3) {
        // |x| <= 3.4e-4: 1 - cos x <= x^2/2 <= 5.8e-8 and (x - sin x)/x <= x^2/6 <= 1.9e-8, both
        // below half an FP32 unit in the last place: cos x = 1 and sin x = x exactly in FP32
        sn = fmaf(k, R, -kref);
        cs = 1.f;
      } else if (SHIFTED == 2) {
        const float x = fmaf(k, R, -kref), xx = x * x;
        cs = fmaf(xx, -0.5f, 1.f);
        sn = fmaf(x * xx, -1.0f / 6.0f, x);
      } else if (SHIFTED == 1) {
        sincos_quarter(fmaf(k, R, -kref), &sn, &cs);
      } else {
        sincos_far(k * R, &sn, &cs);
      }
      const float gw = Q.w[tl][j] * rinv;
      const float gr = gw * cs, gi = gw * sn;
      s0r += gr;
      s0i += gi;
      s1r[0] = fmaf(gr, q.x, s1r[0]);
      s1r[1] = fmaf(gr, q.y, s1r[1]);
      s1r[2] = fmaf(gr, q.z, s1r[2]);
      s1i[0] = fmaf(gi, q.x, s1i[0]);
      s1i[1] = fmaf(gi, q.y, s1i[1]);
      s1i[2] = fmaf(gi, q.z, s1i[2]);
    }
    M.I0r = fmaf(wsi, s0r, M.I0r);
    M.I0i = fmaf(wsi, s0i, M.I0i);
    const float rsi[3] = {rsx, rsy, rsz};
    float dr = 0.f, di = 0.f;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const float wr = wsi * rsi[e];
      M.Ir_r[e] = fmaf(wr, s0r, M.Ir_r[e]);
      M.Ir_i[e] = fmaf(wr, s0i, M.Ir_i[e]);
      M.Ip_r[e] = fmaf(wsi, s1r[e], M.Ip_r[e]);
      M.Ip_i[e] = fmaf(wsi, s1i[e], M.Ip_i[e]);
      dr = fmaf(wr, s1r[e], dr);
      di = fmaf(wr, s1i[e], di);
    }
    M.Irr_r += dr;
    M.Irr_i += di;
  }
  M.Irr_r *= -0.5f;
  M.Irr_i *= -0.5f;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    M.Ip_r[e] *= -0.5f;
    M.Ip_i[e] *= -0.5f;
  }
}

// V and the T_A contributions of one far pair (s outer cell sl of S, t cell tl of Tt)
__device__ __forceinline__ void far_store(const TileCells& S, const TileCells& Tt, int sl, int tl, int s, int t,
                                          const FarMoments& Mo, size_t ldN, size_t ldC, float2* __restrict__ TA,
                                          float2* __restrict__ V) {
  const float inv_aa = S.inv_area[sl] * Tt.inv_area[tl];
  V[(size_t)s * ldC + t] = make_float2(Mo.I0r * inv_aa, Mo.I0i * inv_aa);
  V[(size_t)t * ldC + s] = make_float2(Mo.I0r * inv_aa, Mo.I0i * inv_aa);
  const float quarter = 0.25f * inv_aa;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float ax = S.aloc[sl][3 * a], ay = S.aloc[sl][3 * a + 1], az = S.aloc[sl][3 * a + 2];
    // Irr - a.Irp (shared by the three j)
    const float pa_r = Mo.Irr_r - (ax * Mo.Ip_r[0] + ay * Mo.Ip_r[1] + az * Mo.Ip_r[2]);
    const float pa_i = Mo.Irr_i - (ax * Mo.Ip_i[0] + ay * Mo.Ip_i[1] + az * Mo.Ip_i[2]);
    const int m = S.edge[sl][a];
    if (m < 0) continue;  // a boundary edge of an open surface: no RWG function
    const float sa = S.sign[sl][a] * quarter;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float bx = Tt.aloc[tl][3 * b], by = Tt.aloc[tl][3 * b + 1], bz = Tt.aloc[tl][3 * b + 2];
      const float ab = ax * bx + ay * by + az * bz;
      const float vr = pa_r - (bx * Mo.Ir_r[0] + by * Mo.Ir_r[1] + bz * Mo.Ir_r[2]) + ab * Mo.I0r;
      const float vi = pa_i - (bx * Mo.Ir_i[0] + by * Mo.Ir_i[1] + bz * Mo.Ir_i[2]) + ab * Mo.I0i;
      const float f = sa * Tt.sign[tl][b];
      const int n = Tt.edge[tl][b];
      if (n < 0) continue;
      // T_A is complex symmetric: only the upper triangle is accumulated (m != n on far pairs),
      // the lower one is mirrored afterwards so that both are bit-identical
      atomic_add_c64(&TA[(size_t)min(m, n) * ldN + max(m, n)], f * vr, f * vi);
    }
  }
}

// MINB: resident CTAs per SM that the register allocation is sized for (the plan's choice).
// PATH: the phase treatment, chosen on the host from the quadrature radii.  2: the short series
// for every pair (k (r_s + r_t) <= 1/20 for the largest radii); 4: chosen per pair among no series
// (<= 3.4e-4), the short series, the quarter-turn series and the full reduction, for launches
// where the typical pair needs no series; 0: per pair among the last three (measured on GB300 at
// 20480 cells: 14.04 / 12.65 / 14.11 ms for a launch at ka = 1 / 1e-3 / either).
// Thread (sl, l) of a 32 x 32 tile pair takes s-cell sl against t-cells l, l + 8, l + 16, l + 24.
template <int MINB, int PATH>
__global__ void __launch_bounds__(FAR_THREADS, MINB)
far_pairs_kernel(const DeviceGeometry g, float k, float2* __restrict__ TA, float2* __restrict__ V, int nb) {
  RF_COUNT_LAUNCH();
  __shared__ TileCells S, Tt;
  __shared__ SourceTile Q;
  // linear tile index -> (bi, bj), bi <= bj, row-major over the upper triangle: row bi starts at
  // T(bi) = bi (2 nb - bi + 1) / 2, so bi is the root of T(bi) = tix rounded down, corrected by
  // at most a step either way for the rounding of the square root
  const long long tix = blockIdx.x;
  const double b2 = 2.0 * nb + 1.0;
  int bi = (int)floor(0.5 * (b2 - sqrt(fmax(b2 * b2 - 8.0 * (double)tix, 0.0))));
  bi = max(0, min(bi, nb - 1));
  auto row_start = [nb](long long r) { return r * (2LL * nb - r + 1) / 2; };
  if (row_start(bi) > tix) --bi;
  else if (bi + 1 < nb && row_start(bi + 1) <= tix) ++bi;
  const int bj = bi + (int)(tix - row_start(bi));
  load_tiles(S, Tt, Q, g, bi * TILE, bj * TILE);

  const int sl = threadIdx.x >> 3;
  const int s = bi * TILE + sl;
  if (s >= g.nc) return;
  const size_t ldN = g.ldN, ldC = g.ldC;
  const int NC = g.nc;
  // a fully unrolled source loop hoists its shared-memory reads into registers
  constexpr int UNR = MINB >= 4 ? 2 : 7;

  for (int q = 0; q < 4; ++q) {
    const int tl = (threadIdx.x & 7) + 8 * q;
    const int t = bj * TILE + tl;
    if (t >= NC) continue;
    if (bi == bj && t <= s) continue;
    // near pairs (a shared vertex) belong to the FP64 kernel
    bool near = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) near |= (S.vid[sl][a] == Tt.vid[tl][b]);
    if (near) continue;
    float d[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) d[e] = (S.cen_hi[sl][e] - Tt.cen_hi[tl][e]) + (S.cen_lo[sl][e] - Tt.cen_lo[tl][e]);

    // e^{ikR} = e^{ik Rc} e^{ik (R - Rc)} with Rc the centroid distance: |R - Rc| is at most the
    // sum of the two quadrature radii, so where k times that is within pi/4 the 49 evaluations
    // take sin and cos of k (R - Rc) without a range reduction (a shorter series within 1/20,
    // the common case at low frequency; none at all within 3.4e-4, where cos = 1 and sin x = x
    // to FP32 rounding) and the factor e^{ik Rc} multiplies the eight moments once
    const float dd = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
    const float kRc = k * (dd * rsqrtf(dd));
    const float span = k * (S.rq[sl] + Tt.rq[tl]);  // bound on |k (R - Rc)|
    FarMoments Mo;
    if (PATH == 2) {
      far_moments<2, UNR>(S, sl, Q, tl, d, k, kRc, Mo);
      Mo.rotate(kRc);
    } else {
      if (PATH == 4 && span <= 3.4e-4f) far_moments<3, UNR>(S, sl, Q, tl, d, k, kRc, Mo);
      else if (span <= 0.05f) far_moments<2, UNR>(S, sl, Q, tl, d, k, kRc, Mo);
      else if (span <= 0.78f) far_moments<1, UNR>(S, sl, Q, tl, d, k, kRc, Mo);
      else far_moments<0, UNR>(S, sl, Q, tl, d, k, 0.f, Mo);
      if (span <= 0.78f) Mo.rotate(kRc);
    }
    far_store(S, Tt, sl, tl, s, t, Mo, ldN, ldC, TA, V);
  }
}

// ---------------------------------------------------------------- near pairs (FP64)
struct Pot {
  double S;       // int 1/R
  double V[3];    // int (r' - p)/R
  double p[3];    // projection of r on the plane
};

__device__ __forceinline__ double rpl(double R, double l, double R02) {
  // R + l without cancellation (R >= |l|)
  return l > 0.0 ? R + l : R02 / (R - l);
}

// closed-form integrals over the flat triangle (P0, P1, P2), counter-clockwise
__device__ Pot triangle_potentials(const double r[3], const double* P0, const double* P1, const double* P2) {
  double e1[3], e2[3], n[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = P1[a] - P0[a];
    e2[a] = P2[a] - P0[a];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int a = 0; a < 3; ++a) n[a] /= nn;
  double d = (r[0] - P0[0]) * n[0] + (r[1] - P0[1]) * n[1] + (r[2] - P0[2]) * n[2];
  Pot out;
  for (int a = 0; a < 3; ++a) {
    out.p[a] = r[a] - d * n[a];
    out.V[a] = 0.0;
  }
  out.S = 0.0;
  const double ad = fabs(d);
  const double* P[3] = {P0, P1, P2};
  for (int i = 0; i < 3; ++i) {
    const double* A = P[i];
    const double* B = P[(i + 1) % 3];
    double lv[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double le = sqrt(lv[0] * lv[0] + lv[1] * lv[1] + lv[2] * lv[2]);
    for (int a = 0; a < 3; ++a) lv[a] /= le;
    // outward in-plane normal u = l x n
    double u[3] = {lv[1] * n[2] - lv[2] * n[1], lv[2] * n[0] - lv[0] * n[2], lv[0] * n[1] - lv[1] * n[0]};
    double lp = 0, lm = 0, P0d = 0;
    for (int a = 0; a < 3; ++a) {
      lp += (B[a] - out.p[a]) * lv[a];
      lm += (A[a] - out.p[a]) * lv[a];
      P0d += (A[a] - out.p[a]) * u[a];
    }
    const double R02 = P0d * P0d + d * d;
    const double Rp = sqrt(lp * lp + R02), Rm = sqrt(lm * lm + R02);
    double F = 0.0;
    if (R02 > 1e-30 * le * le) F = log(rpl(Rp, lp, R02) / rpl(Rm, lm, R02));
    double at = 0.0;
    if (ad > 0.0) at = atan2(P0d * lp, R02 + ad * Rp) - atan2(P0d * lm, R02 + ad * Rm);
    out.S += P0d * F - ad * at;
    const double c = 0.5 * (R02 * F + lp * Rp - lm * Rm);
    for (int a = 0; a < 3; ++a) out.V[a] += c * u[a];
  }
  return out;
}

constexpr int NEAR_PAIRS_PER_BLOCK = 8;
constexpr int NEAR_THREADS = NEAR_PAIRS_PER_BLOCK * 16;

// 16 slots per pair: slot = order * 7 + outer point, slots 14, 15 idle
__global__ void __launch_bounds__(NEAR_THREADS)
near_pairs_kernel(const DeviceGeometry g, double k, float2* __restrict__ TA, float2* __restrict__ V) {
  RF_COUNT_LAUNCH();
  __shared__ double mom[NEAR_PAIRS_PER_BLOCK][16][16];  // per slot: I0(2) Iouter(6) Iinner(6) Irr(2)
  const int lp = threadIdx.x >> 4;
  const int slot = threadIdx.x & 15;
  const int pair = blockIdx.x * NEAR_PAIRS_PER_BLOCK + lp;
  double acc[16];
  for (int e = 0; e < 16; ++e) acc[e] = 0.0;
  if (pair < g.n_near && slot < 14) {
    const int order = slot / 7, i = slot % 7;
    const int s = g.near_pairs[2 * pair], t = g.near_pairs[2 * pair + 1];
    const int so = order == 0 ? s : t;  // outer (test) cell
    const int si = order == 0 ? t : s;  // inner (source) cell
    double r[3], rho_o[3];
    for (int a = 0; a < 3; ++a) {
      r[a] = g.qp64[21 * so + 3 * i + a];
      rho_o[a] = r[a] - g.cen64[3 * so + a];
    }
    const double* P0 = g.verts + 3 * g.tris[3 * si];
    const double* P1 = g.verts + 3 * g.tris[3 * si + 1];
    const double* P2 = g.verts + 3 * g.tris[3 * si + 2];
    Pot pt = triangle_potentials(r, P0, P1, P2);
    // singular part: J0 = S / 4pi, J1 = (Vv + (p - c_si) S) / 4pi (relative to the inner centroid)
    double J0r = pt.S * INV_4PI, J0i = 0.0;
    double J1r[3], J1i[3];
    for (int a = 0; a < 3; ++a) {
      J1r[a] = (pt.V[a] + (pt.p[a] - g.cen64[3 * si + a]) * pt.S) * INV_4PI;
      J1i[a] = 0.0;
    }
    // smooth part (e^{ikR} - 1)/(4 pi R) on the inner 7-point rule, value i k / 4pi at R = 0.  It
    // is bounded and smooth (real part -2 sin^2(kR/2) / (4 pi R), imaginary sin(kR) / (4 pi R)),
    // so it runs in FP32 from the centroid-local quadrature offsets (GB300's FP64 pipe is slow),
    // added to the FP64 singular part once per point
    {
      const float kf = (float)k;
      float dc[3], ro[3];
      for (int a = 0; a < 3; ++a) {
        dc[a] = (g.cen_hi[3 * so + a] - g.cen_hi[3 * si + a]) + (g.cen_lo[3 * so + a] - g.cen_lo[3 * si + a]);
        ro[a] = g.rho[21 * so + 3 * i + a];
      }
      float s0r = 0.f, s0i = 0.f, s1r[3] = {0.f, 0.f, 0.f}, s1i[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        float ri[3], R2 = 0.f;
        for (int a = 0; a < 3; ++a) {
          ri[a] = g.rho[21 * si + 3 * j + a];
          const float dd = dc[a] + (ro[a] - ri[a]);
          R2 = fmaf(dd, dd, R2);
        }
        float gr, gi;
        if (so == si && j == i) {  // the same point (R = 0 exactly)
          gr = 0.f;
          gi = kf * INV_4PI_F;
        } else {
          const float rinv = rsqrtf(R2);
          float sh, ch;
          sincos_far(0.5f * kf * (R2 * rinv), &sh, &ch);
          gr = -2.f * sh * sh * INV_4PI_F * rinv;
          gi = 2.f * sh * ch * INV_4PI_F * rinv;
        }
        const float w = g.wq[7 * si + j];
        s0r = fmaf(w, gr, s0r);
        s0i = fmaf(w, gi, s0i);
        for (int a = 0; a < 3; ++a) {
          s1r[a] = fmaf(w * gr, ri[a], s1r[a]);
          s1i[a] = fmaf(w * gi, ri[a], s1i[a]);
        }
      }
      J0r += (double)s0r;
      J0i += (double)s0i;
      for (int a = 0; a < 3; ++a) {
        J1r[a] += (double)s1r[a];
        J1i[a] += (double)s1i[a];
      }
    }
    const double wo = (i == 0 ? 9.0 / 40.0 : (i < 4 ? (155.0 - sqrt(15.0)) / 1200.0 : (155.0 + sqrt(15.0)) / 1200.0)) *
                      g.area64[so];
    acc[0] = wo * J0r;
    acc[1] = wo * J0i;
    double dr = 0.0, di = 0.0;
    for (int a = 0; a < 3; ++a) {
      acc[2 + a] = wo * rho_o[a] * J0r;   // outer moment
      acc[5 + a] = wo * rho_o[a] * J0i;
      acc[8 + a] = wo * J1r[a];           // inner moment
      acc[11 + a] = wo * J1i[a];
      dr += rho_o[a] * J1r[a];
      di += rho_o[a] * J1i[a];
    }
    acc[14] = wo * dr;
    acc[15] = wo * di;
  }
  for (int e = 0; e < 16; ++e) mom[lp][slot][e] = acc[e];
  __syncthreads();
  if (slot != 0 || pair >= g.n_near) return;
  // sum each order over its 7 points, then average the two orders in the (s, t) frame
  double o0[16], o1[16];
  for (int e = 0; e < 16; ++e) {
    o0[e] = 0.0;
    o1[e] = 0.0;
    for (int i = 0; i < 7; ++i) {
      o0[e] += mom[lp][i][e];
      o1[e] += mom[lp][7 + i][e];
    }
  }
  const int s = g.near_pairs[2 * pair], t = g.near_pairs[2 * pair + 1];
  double I0r = 0.5 * (o0[0] + o1[0]), I0i = 0.5 * (o0[1] + o1[1]);
  double Isr[3], Isi[3], Itr[3], Iti[3];
  for (int a = 0; a < 3; ++a) {
    Isr[a] = 0.5 * (o0[2 + a] + o1[8 + a]);  // int rho_s G
    Isi[a] = 0.5 * (o0[5 + a] + o1[11 + a]);
    Itr[a] = 0.5 * (o0[8 + a] + o1[2 + a]);  // int rho_t G
    Iti[a] = 0.5 * (o0[11 + a] + o1[5 + a]);
  }
  double Irr_r = 0.5 * (o0[14] + o1[14]), Irr_i = 0.5 * (o0[15] + o1[15]);
  const size_t ldN = g.ldN, ldC = g.ldC;
  const double inv_aa = 1.0 / (g.area64[s] * g.area64[t]);
  V[(size_t)s * ldC + t] = make_float2((float)(I0r * inv_aa), (float)(I0i * inv_aa));
  if (s != t) V[(size_t)t * ldC + s] = make_float2((float)(I0r * inv_aa), (float)(I0i * inv_aa));
  for (int a = 0; a < 3; ++a) {
    double ai[3], pr = Irr_r, pi = Irr_i;
    for (int x = 0; x < 3; ++x) {
      ai[x] = g.verts[3 * g.tris[3 * s + a] + x] - g.cen64[3 * s + x];
      pr -= ai[x] * Itr[x];
      pi -= ai[x] * Iti[x];
    }
    const int m = g.cell_edges[3 * s + a];
    if (m < 0) continue;  // a boundary edge of an open surface: no RWG function
    const double sa = (double)g.cell_sign[3 * s + a] * 0.25 * inv_aa;
    for (int b = 0; b < 3; ++b) {
      double vr = pr, vi = pi, ab = 0.0;
      for (int x = 0; x < 3; ++x) {
        const double bx = g.verts[3 * g.tris[3 * t + b] + x] - g.cen64[3 * t + x];
        vr -= bx * Isr[x];
        vi -= bx * Isi[x];
        ab += ai[x] * bx;
      }
      vr += ab * I0r;
      vi += ab * I0i;
      const double f = sa * (double)g.cell_sign[3 * t + b];
      const int n = g.cell_edges[3 * t + b];
      if (n < 0) continue;
      // upper triangle only: a distinct pair reaches (m, n) and (n, m) once each, which is
      // twice on the diagonal; the self pair lists both (a, b) and (b, a) itself
      double mult = 1.0;
      if (s != t) {
        if (m == n) mult = 2.0;
      } else if (m > n) {
        mult = 0.0;
      }
      if (mult != 0.0)
        atomic_add_c64(&TA[(size_t)min(m, n) * ldN + max(m, n)], (float)(mult * f * vr), (float)(mult * f * vi));
    }
  }
}

// ---------------------------------------------------------------- mirror upper -> lower
constexpr int MT = 32;

__global__ void mirror_upper_kernel(float2* __restrict__ M, int n, size_t ld) {
  RF_COUNT_LAUNCH();
  // block (bx, by) with by <= bx copies tile (by, bx) of the upper triangle into tile (bx, by)
  __shared__ float2 tile[MT][MT + 1];
  const int bx = blockIdx.x, by = blockIdx.y;
  if (by > bx) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < MT; r += 8) {
    const int row = by * MT + r, col = bx * MT + tx;
    if (row < n && col < n && row < col) tile[r][tx] = M[(size_t)row * ld + col];
  }
  __syncthreads();
  for (int r = ty; r < MT; r += 8) {
    const int row = bx * MT + r, col = by * MT + tx;  // lower entry (row, col) = upper (col, row)
    if (row < n && col < n && col < row) M[(size_t)row * ld + col] = tile[tx][r];
  }
}

// ---------------------------------------------------------------- excitation (FP64)
// Delta-gap excitation: the edges whose two cells have their centroids on opposite sides of the
// plane (o, u) carry e_n = +-V (the flux of an RWG function through its own edge is 1), + where
// c^+ lies on the negative side; every other edge 0.
__global__ void gap_kernel(const DeviceGeometry g, double ox, double oy, double oz, double ux, double uy, double uz,
                           double vr, double vi, double2* __restrict__ e) {
  RF_COUNT_LAUNCH();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.ne) return;
  const double* cp = g.cen64 + 3 * g.edge_cells[2 * n];
  const double* cm = g.cen64 + 3 * g.edge_cells[2 * n + 1];
  const bool sp = (cp[0] - ox) * ux + (cp[1] - oy) * uy + (cp[2] - oz) * uz > 0.0;
  const bool sm = (cm[0] - ox) * ux + (cm[1] - oy) * uy + (cm[2] - oz) * uz > 0.0;
  const double s = sp == sm ? 0.0 : (sp ? -1.0 : 1.0);
  e[n] = make_double2(s * vr, s * vi);
}

__global__ void rhs_kernel(const DeviceGeometry g, double k, const double* __restrict__ khat,
                           const double* __restrict__ pol, int nrhs, double2* __restrict__ e) {
  RF_COUNT_LAUNCH();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (n >= g.ne || r >= nrhs) return;
  const double kx = khat[3 * r], ky = khat[3 * r + 1], kz = khat[3 * r + 2];
  const double px = pol[3 * r], py = pol[3 * r + 1], pz = pol[3 * r + 2];
  double accr = 0.0, acci = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int c = g.edge_cells[2 * n + side];
    const int fv = g.edge_free[2 * n + side];
    const double sg = side == 0 ? 0.5 : -0.5;  // sigma / (2 A) times the area of the rule
    for (int q = 0; q < 7; ++q) {
      const double* rq = g.qp64 + 21 * c + 3 * q;
      const double w = q == 0 ? 9.0 / 40.0 : (q < 4 ? (155.0 - sqrt(15.0)) / 1200.0 : (155.0 + sqrt(15.0)) / 1200.0);
      const double dot = (rq[0] - g.verts[3 * fv]) * px + (rq[1] - g.verts[3 * fv + 1]) * py +
                         (rq[2] - g.verts[3 * fv + 2]) * pz;
      double sn, cs;
      sincos(k * (kx * rq[0] + ky * rq[1] + kz * rq[2]), &sn, &cs);
      accr += sg * w * dot * cs;
      acci += sg * w * dot * sn;
    }
  }
  e[(size_t)r * g.ne + n] = make_double2(accr, acci);
}

// ---------------------------------------------------------------- radiation vector (FP64)
// F(u) = sum_cells sum_q w_q e^{-ik u.r_q} J_c(r_q) over the 7-point rule, with the cell current
// J_c(r) = sum_i s_i j_i (r - P_i) / 2 (the RWG functions of Eq. RWGdef times the cell area of
// the product rule) = (r S - T) / 2, S = sum_i s_i j_i, T = sum_i s_i j_i P_i.  Hence
//   F_c = (S B1 - T B0) / 2,  B0 = sum_q w_q e^{-ik u.r_q},  B1 = sum_q w_q e^{-ik u.r_q} r_q,
// where B0 and B1 depend on the direction and the cell only (one set for RB right-hand sides),
// and e^{-ik u.r_q} = e^{-ik u.c} e^{-ik u.(r_q - c)} (c the centroid) takes one sincos per cell
// and, per point, the Taylor series of a small angle.  Everything stays FP64: at low frequency
// the radiated field is a small remainder of the cell contributions.
constexpr int FF_THREADS = 256;

// cos and sin of |x| <= 1/20 by their Taylor series (to x^6 and x^7: truncation below 1e-15)
__device__ __forceinline__ void sincos_tiny64(double x, double* s, double* c) {
  const double x2 = x * x;
  *c = fma(x2, fma(x2, fma(x2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  *s = fma(x * x2, fma(x2, fma(x2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), x);
}

// cos and sin of |x| <= 1/2 by their Taylor series (to x^12 and x^13: truncation below 1e-15)
__device__ __forceinline__ void sincos_small64(double x, double* s, double* c) {
  const double x2 = x * x;
  double pc = fma(x2, 1.0 / 479001600.0, -1.0 / 3628800.0);
  pc = fma(x2, pc, 1.0 / 40320.0);
  pc = fma(x2, pc, -1.0 / 720.0);
  pc = fma(x2, pc, 1.0 / 24.0);
  pc = fma(x2, pc, -0.5);
  *c = fma(x2, pc, 1.0);
  double ps = fma(x2, 1.0 / 6227020800.0, -1.0 / 39916800.0);
  ps = fma(x2, ps, 1.0 / 362880.0);
  ps = fma(x2, ps, -1.0 / 5040.0);
  ps = fma(x2, ps, 1.0 / 120.0);
  ps = fma(x2, ps, -1.0 / 6.0);
  *s = fma(x * x2, ps, x);
}

template <int RB>
__global__ void __launch_bounds__(FF_THREADS)
farfield_kernel(const DeviceGeometry g, double k, const double2* __restrict__ j, int nrhs, const double* dirs,
                int ndir, double2* __restrict__ out) {
  RF_COUNT_LAUNCH();
  const int d = blockIdx.x;
  const int r0 = blockIdx.y * RB;
  const double ux = dirs[3 * d], uy = dirs[3 * d + 1], uz = dirs[3 * d + 2];
  // 7-point rule weights (sum 1) times 1/2
  const double wa = 0.5 * (9.0 / 40.0), wb = 0.5 * (155.0 - 3.872983346207416885) / 1200.0,
               wc = 0.5 * (155.0 + 3.872983346207416885) / 1200.0;
  double acc[RB][6];
#pragma unroll
  for (int b = 0; b < RB; ++b)
#pragma unroll
    for (int e = 0; e < 6; ++e) acc[b][e] = 0.0;
  for (int c = threadIdx.x; c < g.nc; c += blockDim.x) {
    const double cx = g.cen64[3 * c], cy = g.cen64[3 * c + 1], cz = g.cen64[3 * c + 2];
    double b0r = 0.0, b0i = 0.0, b1r[3] = {0.0, 0.0, 0.0}, b1i[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const double* rq = g.qp64 + 21 * c + 3 * q;
      const double x = -k * (ux * (rq[0] - cx) + uy * (rq[1] - cy) + uz * (rq[2] - cz));
      double sn, cs;
      const double ax = fabs(x);
      if (ax <= 0.05) sincos_tiny64(x, &sn, &cs);
      else if (ax <= 0.5) sincos_small64(x, &sn, &cs);
      else sincos(x, &sn, &cs);
      const double w = q == 0 ? wa : (q < 4 ? wb : wc);
      const double er = w * cs, ei = w * sn;
      b0r += er;
      b0i += ei;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        b1r[e] = fma(er, rq[e], b1r[e]);
        b1i[e] = fma(ei, rq[e], b1i[e]);
      }
    }
    {  // times e^{-ik u.c}
      double sn, cs;
      sincos(-k * (ux * cx + uy * cy + uz * cz), &sn, &cs);
      double t = b0r;
      b0r = t * cs - b0i * sn;
      b0i = t * sn + b0i * cs;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        t = b1r[e];
        b1r[e] = t * cs - b1i[e] * sn;
        b1i[e] = t * sn + b1i[e] * cs;
      }
    }
    int ed[3];
    double sg[3];
    const double* P[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ed[i] = g.cell_edges[3 * c + i];
      sg[i] = (double)g.cell_sign[3 * c + i];
      P[i] = g.verts + 3 * g.tris[3 * c + i];
    }
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (r0 + b >= nrhs) break;
      const double2* jr = j + (size_t)(r0 + b) * g.ne;
      double sr = 0.0, si = 0.0, tr[3] = {0.0, 0.0, 0.0}, ti[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (ed[i] < 0) continue;  // a boundary edge: no current
        const double2 v = jr[ed[i]];
        const double vr = sg[i] * v.x, vi = sg[i] * v.y;
        sr += vr;
        si += vi;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          tr[e] = fma(vr, P[i][e], tr[e]);
          ti[e] = fma(vi, P[i][e], ti[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < 3; ++e) {  // S B1 - T B0
        acc[b][2 * e] += (sr * b1r[e] - si * b1i[e]) - (tr[e] * b0r - ti[e] * b0i);
        acc[b][2 * e + 1] += (sr * b1i[e] + si * b1r[e]) - (tr[e] * b0i + ti[e] * b0r);
      }
    }
  }
  __shared__ double red[FF_THREADS / 32][6];
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    if (r0 + b >= nrhs) break;
    for (int e = 0; e < 6; ++e) {
      double v = acc[b][e];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][e] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      double v = 0.0;
      for (int w = 0; w < FF_THREADS / 32; ++w) v += red[w][threadIdx.x];
      double* o = reinterpret_cast<double*>(out + ((size_t)(r0 + b) * ndir + d) * 3);
      o[threadIdx.x] = v;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_assemble_far(const DeviceGeometry& g, float k, float2* TA, float2* V, int min_blocks,
                                cudaStream_t s) {
  const int nb = (g.nc + TILE - 1) / TILE;
  const long long tiles = (long long)nb * (nb + 1) / 2;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  // far pairs: all unordered pairs minus the near ones (n_near counts s <= t, including s == t)
  const double far = (double)g.nc * (g.nc + 1) / 2.0 - (double)g.n_near;
  ProfScope prof("assemble_far", 8.0 * (double)g.nc * g.nc + 8.0 * (double)g.ne * g.ne, far * 49.0 * 54.0, s);
  // every pair's phase span k (r_s + r_t) is at most 2 k rq_max; a typical pair's about 2 k rq_mean
  const double span_max = 2.0 * (double)k * (double)g.rq_max, span_mean = 2.0 * (double)k * (double)g.rq_mean;
  const int path = span_mean <= 3.4e-4 ? 4 : (span_max <= 0.05 ? 2 : 0);
#define RF_FAR(MB)                                                                           \
  if (path == 4) far_pairs_kernel<MB, 4><<<(unsigned)tiles, FAR_THREADS, 0, s>>>(g, k, TA, V, nb); \
  else if (path == 2) far_pairs_kernel<MB, 2><<<(unsigned)tiles, FAR_THREADS, 0, s>>>(g, k, TA, V, nb); \
  else far_pairs_kernel<MB, 0><<<(unsigned)tiles, FAR_THREADS, 0, s>>>(g, k, TA, V, nb);
  switch (min_blocks) {
    case 1:
      RF_FAR(1)
      break;
    case 2:
      RF_FAR(2)
      break;
    case 0:
    case 3:
      RF_FAR(3)
      break;
    case 4:
      RF_FAR(4)
      break;
    default:
      return cudaErrorInvalidValue;
  }
#undef RF_FAR
  return cudaGetLastError();
}

cudaError_t launch_assemble_near(const DeviceGeometry& g, double k, float2* TA, float2* V, cudaStream_t s) {
  if (g.n_near == 0) return cudaSuccess;
  const int blocks = (g.n_near + NEAR_PAIRS_PER_BLOCK - 1) / NEAR_PAIRS_PER_BLOCK;
  ProfScope prof("assemble_near", 0.0, 0.0, s);
  near_pairs_kernel<<<blocks, NEAR_THREADS, 0, s>>>(g, k, TA, V);
  return cudaGetLastError();
}

cudaError_t launch_mirror_upper(float2* M, int n, int ld, cudaStream_t s) {
  const int nb = (n + MT - 1) / MT;
  dim3 grid(nb, nb), block(MT, 8);
  ProfScope prof("mirror_upper", 8.0 * (double)n * n, 0.0, s);
  mirror_upper_kernel<<<grid, block, 0, s>>>(M, n, (size_t)ld);
  return cudaGetLastError();
}

cudaError_t launch_rhs_voltage_gap(const DeviceGeometry& g, const double* origin, const double* normal, double2 v,
                                   double2* e, cudaStream_t s) {
  const double nn = std::sqrt(normal[0] * normal[0] + normal[1] * normal[1] + normal[2] * normal[2]);
  gap_kernel<<<(g.ne + 255) / 256, 256, 0, s>>>(g, origin[0], origin[1], origin[2], normal[0] / nn, normal[1] / nn,
                                                normal[2] / nn, v.x, v.y, e);
  return cudaGetLastError();
}

cudaError_t launch_rhs_planewave(const DeviceGeometry& g, double k, const double* khat, const double* pol, int nrhs,
                                 double2* e, cudaStream_t s) {
  dim3 grid((g.ne + 255) / 256, nrhs);
  rhs_kernel<<<grid, 256, 0, s>>>(g, k, khat, pol, nrhs, e);
  return cudaGetLastError();
}

cudaError_t launch_farfield(const DeviceGeometry& g, double k, const double2* j, int nrhs, const double* dirs,
                            int ndir, double2* out, cudaStream_t s) {
  ProfScope prof("farfield", 0.0, 0.0, s);
  if (nrhs == 1) {
    farfield_kernel<1><<<dim3(ndir, 1), FF_THREADS, 0, s>>>(g, k, j, nrhs, dirs, ndir, out);
  } else {
    farfield_kernel<4><<<dim3(ndir, (nrhs + 3) / 4), FF_THREADS, 0, s>>>(g, k, j, nrhs, dirs, ndir, out);
  }
  return cudaGetLastError();
}

RF_LAUNCH_READER(launches_assembly)

}  // namespace rfcmp
