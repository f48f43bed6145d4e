// Per-tile front-to-back alpha compositing (forward) and its reverse-order
// backward pass.
//
// 3D-GS composites each pixel over its tile's depth-sorted list (the paper
// trains that renderer, Section I/III): alpha = min(0.99, opacity *
// exp(power)), skip if power > 0 or alpha < 1/255, stop before a Gaussian
// that would bring T below 1e-4.  The backward pass walks the same list from
// each pixel's last contributor towards the front, recovering T by division
// and keeping the colour composited behind.
//
// Launch shapes, selected per context (GS_OPT_RASTER_FWD / _BWD): PPT = 1, 2
// or 4 pixels per thread with 8, 4 or 2 warps per tile (each warp an 8-pixel-
// wide band), or PPT = 8 with one warp per 16x16 tile.  Every warp walks its
// tile's list independently (no block barriers).  It stages 32 records at a
// time, one per lane; each lane tests its record's alpha >= 1/255 ellipse
// (with a rounding margin) against the warp's pixel rectangle, and the warp
// walks only the survivors (a ballot mask); with 2 pixels per thread the
// warp's lanes form groups that each walk the records whose alpha >= 1/255
// box reaches their own sub-rectangle (see LaneGroups; no ellipse test).
// This removes only pairs that the per-pixel test would skip, so the result
// is unchanged.
#include "gs_internal.cuh"
#include "launch.h"

namespace gs {

__device__ __forceinline__ int view_of_bin(const ViewRec* views, int B, int bin) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_offset <= bin) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Staged Gaussian (shared memory, three float4), as written by the projection:
//   s0 = (mu_x, mu_y, cA, cB), s1 = (cC, opacity, r, g), s2 = (b, hx, hy, depth)
// with p2 = cA dx^2 + cB dx dy + cC dy^2 = power * log2(e), dx = mu_x - x,
// and (hx, hy) the half-extents of the box around the alpha >= 1/255 ellipse.
__device__ __forceinline__ void stage_one(const RasterArgs& a, int v, uint32_t g, float4& s0, float4& s1,
                                          float4& s2) {
  if ((int64_t)g >= a.n) {  // only after a capacity overflow: a box nothing hits
    s0 = make_float4(0.f, 0.f, 0.f, 0.f);
    s1 = s0;
    s2 = make_float4(0.f, -3.0e38f, -3.0e38f, 0.f);
    return;
  }
  const int64_t o = (int64_t)v * a.stride + g;
  s0 = a.rec0[kRecStride * o];
  s1 = a.rec1[kRecStride * o];
  s2 = a.rec2[kRecStride * o];
}

// Does the splat's alpha >= 1/255 box meet the pixel rectangle [x0,x1]x[y0,y1]?
__device__ __forceinline__ bool box_hits(const float4& s0, const float4& s2, float x0, float x1, float y0,
                                         float y1) {
  return s0.x + s2.y >= x0 && s0.x - s2.y <= x1 && s0.y + s2.z >= y0 && s0.y - s2.z <= y1;
}

// Can any pixel of the rectangle [x0,x1]x[y0,y1] pass the alpha >= 1/255
// test?  p2(u, w) = cA u^2 + cB u w + cC w^2 (u = mu_x - x, w = mu_y - y) is
// concave, so its maximum over the rectangle is 0 when the mean lies inside
// and otherwise lies on an edge, where it is the 1-D maximum at the clamped
// stationary point.  A pixel passes only if opacity * 2^p2 >= 1/255, i.e.
// p2 >= -log2(255 opacity); the threshold is lowered by a margin that covers
// the rounding of the per-pixel FP32 evaluation (relative to the largest term
// magnitude over the rectangle) and of ex2.approx, so the test only removes
// pairs the per-pixel test would skip.
struct EllipseTerms {
  float cA, cB, cC, kw, ku, base;
};

__device__ __forceinline__ EllipseTerms ellipse_terms(const float4& r0, const float4& r1) {
  EllipseTerms t;
  t.cA = r0.z;
  t.cB = r0.w;
  t.cC = r1.x;
  // stationary w for a fixed u and u for a fixed w (an approximate quotient
  // only moves the evaluation point, which changes p2 to second order)
  t.kw = __fdividef(-0.5f * t.cB, t.cC);
  t.ku = __fdividef(-0.5f * t.cB, t.cA);
  const float thr = -__log2f(255.f * r1.y);
  t.base = thr - (1e-3f + 1e-3f * fabsf(thr));
  return t;
}

__device__ __forceinline__ bool ellipse_rect(const EllipseTerms& t, const float4& r0, const float4& r2, float x0,
                                             float x1, float y0, float y1) {
  if (!box_hits(r0, r2, x0, x1, y0, y1)) return false;
  const float u0 = r0.x - x1, u1 = r0.x - x0, w0 = r0.y - y1, w1 = r0.y - y0;
  if (u0 <= 0.f && u1 >= 0.f && w0 <= 0.f && w1 >= 0.f) return true;
  float best = -3.0e38f;
#pragma unroll
  for (int e = 0; e < 2; e++) {
    const float u = e ? u1 : u0;
    const float w = fminf(fmaxf(t.kw * u, w0), w1);
    best = fmaxf(best, fmaf(t.cA * u, u, fmaf(t.cB * u, w, t.cC * w * w)));
    const float w2 = e ? w1 : w0;
    const float u2 = fminf(fmaxf(t.ku * w2, u0), u1);
    best = fmaxf(best, fmaf(t.cA * u2, u2, fmaf(t.cB * u2, w2, t.cC * w2 * w2)));
  }
  const float U = fmaxf(fabsf(u0), fabsf(u1)), W = fmaxf(fabsf(w0), fabsf(w1));
  const float mag = fabsf(t.cA) * U * U + fabsf(t.cB) * U * W + fabsf(t.cC) * W * W;
  return best >= t.base - 1e-5f * mag;
}

__device__ __forceinline__ bool ellipse_hits(const float4& r0, const float4& r1, const float4& r2, float x0,
                                             float x1, float y0, float y1) {
  if (!box_hits(r0, r2, x0, x1, y0, y1)) return false;
  return ellipse_rect(ellipse_terms(r0, r1), r0, r2, x0, x1, y0, y1);
}

// Lane-group survivors: the alpha >= 1/255 box against each group's
// rectangle (bit g: group g).  The box is looser than the ellipse but costs
// four compares per group; the exact ellipse test against the warp's
// rectangle on top of it cost the forward more (its per-record terms) than
// the walk steps it saved.
template <class Geom>
__device__ __forceinline__ uint32_t box_group_bits(const float4& r0, const float4& r2, const Geom& geo) {
  uint32_t bits = 0;
#pragma unroll
  for (int g = 0; g < Geom::NG; g++) {
    float x0, x1, y0, y1;
    geo.group_rect(g, x0, x1, y0, y1);
    bits |= box_hits(r0, r2, x0, x1, y0, y1) ? 1u << g : 0u;
  }
  return bits;
}

// p2 at row offset dy = mu_y - y for a lane with column coefficients
// a0 = cA dx^2, a1 = cB dx.  Every kernel variant, forward and backward,
// evaluates it with the same instructions on the same operands for a given
// pixel, so their skip decisions agree.
__device__ __forceinline__ float splat_p2(float cC, float a1, float a0, float dy) {
  return __fmaf_rn(__fmaf_rn(cC, dy, a1), dy, a0);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float splat_alpha2(float op, float p2, float& G) {
  G = ex2_approx(p2);
  return fminf(kAlphaClamp, __fmul_rn(op, G));
}

// Accumulators hold d/d(mu_x, mu_y) of p2 and raw dx^2, dx dy, dy^2 sums;
// the scale of value q undoes those scalings.
__device__ __forceinline__ float grad_scale(int q) {
  return q < 2 ? (1.f / kLog2e) : (q == 2 || q == 4) ? -0.5f : (q == 3 ? -1.f : 1.f);
}

// The 2D gradient of a (view, Gaussian) pair is a 32-byte geometry record
// dL/d(mu_x, mu_y, A, B), dL/d(C, opacity), 0, 0 and a 16-byte colour
// record dL/d(r, g, b), 0, added with vector reductions (one L2 request per
// 16 or 8 bytes instead of one per value).
__device__ __forceinline__ void red_v4(float* p, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
__device__ __forceinline__ void red_v2(float* p, float x, float y) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ void push_record(float* geo, float* col, const float (&acc)[16]) {
  red_v4(geo, acc[0] * grad_scale(0), acc[1] * grad_scale(1), acc[2] * grad_scale(2), acc[3] * grad_scale(3));
  red_v2(geo + 4, acc[4] * grad_scale(4), acc[5] * grad_scale(5));
  red_v4(col, acc[6], acc[7], acc[8], 0.f);
}

// Apply the gradient of one Gaussian from lane groups of GW lanes that each
// walk their own Gaussian (lane groups aligned to GW; `contrib` is the
// warp's ballot of the lanes whose pixels contributed).  When every group
// has at most direct_max such lanes, those lanes add their own values (3
// reductions each); otherwise each group sums its 9 values over its lanes
// (reduce-scatter for values 0..7, a butterfly for value 8), gathers them
// into two lanes and adds the totals (3 reductions per group).
template <int GW>
__device__ __forceinline__ void push_grad_group(float* g2d, int64_t entries, int64_t rec, float (&acc)[16], int lane,
                                                uint32_t contrib, int direct_max) {
  static_assert(GW == 4 || GW == 8 || GW == 16 || GW == 32, "lane groups of 4, 8, 16 or 32");
  float* const r = g2d + kG2dGeo * rec;                         // geometry record
  float* const rc = g2d + kG2dGeo * entries + kG2dCol * rec;    // colour record
  const int gl = lane % GW;
  const uint32_t gbits = GW == 32 ? contrib : (contrib >> (lane - gl)) & ((1u << (GW % 32)) - 1u);
  if (__all_sync(0xffffffffu, __popc(gbits) <= direct_max)) {
    if (contrib & (1u << lane)) push_record(r, rc, acc);
    return;
  }
  if constexpr (GW == 4) {
    // two reduce-scatter levels: lane (b1, b0) of the group holds values
    // 4 b1 + 2 b0 and 4 b1 + 2 b0 + 1
#pragma unroll
    for (int off = 2, half = 4; off >= 1; off >>= 1, half >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < half; i++) {
        const float send = up ? acc[i] : acc[i + half];
        const float keep = up ? acc[i + half] : acc[i];
        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    float t8 = acc[8];
    t8 += __shfl_xor_sync(0xffffffffu, t8, 2);
    t8 += __shfl_xor_sync(0xffffffffu, t8, 1);
    // lanes 0 and 2 of the group take their right neighbour's pair
    const float h0 = __shfl_down_sync(0xffffffffu, acc[0], 1);
    const float h1 = __shfl_down_sync(0xffffffffu, acc[1], 1);
    if (gbits) {
      if (gl == 0) red_v4(r, acc[0] * grad_scale(0), acc[1] * grad_scale(1), h0 * grad_scale(2), h1 * grad_scale(3));
      if (gl == 2) {
        red_v2(r + 4, acc[0] * grad_scale(4), acc[1] * grad_scale(5));
        red_v4(rc, h0, h1, t8, 0.f);
      }
    }
  } else {
#pragma unroll
    for (int off = GW / 2, half = 4; half >= 1; off >>= 1, half >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < half; i++) {
        const float send = up ? acc[i] : acc[i + half];
        const float keep = up ? acc[i + half] : acc[i];
        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    constexpr int S = GW / 8;  // lanes holding each of values 0..7
    float t = acc[0], t8 = acc[8];
#pragma unroll
    for (int off = S / 2; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
#pragma unroll
    for (int off = GW / 2; off >= 1; off >>= 1) t8 += __shfl_xor_sync(0xffffffffu, t8, off);
    // lane 0 of the group gathers values 0..3, lane 4 S values 4..7
    const int src = (lane - gl) + (gl >= 4 * S ? 4 * S : 0);
    float x[4];
#pragma unroll
    for (int k = 0; k < 4; k++) x[k] = __shfl_sync(0xffffffffu, t, src + k * S);
    if (gbits) {
      if (gl == 0) red_v4(r, x[0] * grad_scale(0), x[1] * grad_scale(1), x[2] * grad_scale(2), x[3] * grad_scale(3));
      if (gl == 4 * S) {
        red_v2(r + 4, x[0] * grad_scale(4), x[1] * grad_scale(5));
        red_v4(rc, x[2], x[3], t8, 0.f);
      }
    }
  }
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One backward (pixel, Gaussian) pair, branch-free so that the pixels of a
// thread interleave.  `live` says the pair lies before the pixel's last
// contributor.  T is the transmittance behind the Gaussian on entry and in
// front of it on exit; dCS = sum_c dL/dC_c S_c with S the colour composited
// behind.  Skipped pairs leave every value unchanged.  Returns whether the
// pair contributed.
__device__ __forceinline__ bool bwd_pair(bool live, const float4& q0, const float4& q1, const float (&rgb)[3],
                                         float a0, float a1, float dy, float dx, float dx2, float cA2dx, float cBdx,
                                         float& T, float& dCS, const float (&dC)[3], float bgd, float (&acc)[16]) {
  const float p2 = splat_p2(q1.x, a1, a0, dy);
  float G;
  const float alpha = splat_alpha2(q1.y, p2, G);
  const bool on = live && !(p2 > 0.f) && !(alpha < kAlphaSkip);
  const float ae = on ? alpha : 0.f;
  // 1 - ae is in [0.01, 1]: the approximate reciprocal (relative error
  // below 2^-22) keeps the recovered T within FP32 rounding of the division
  const float inv_om = rcp_approx(1.f - ae);
  const float Ti = T * inv_om;
  const float wgt = ae * Ti;
  const float dcr = dC[0] * rgb[0] + dC[1] * rgb[1] + dC[2] * rgb[2];
  const float dLda = Ti * dcr - inv_om * (bgd + dCS);
  acc[6] = fmaf(dC[0], wgt, acc[6]);
  acc[7] = fmaf(dC[1], wgt, acc[7]);
  acc[8] = fmaf(dC[2], wgt, acc[8]);
  dCS = fmaf(wgt, dcr, dCS);
  T = Ti;
  // zero through a clamped alpha (opacity G > 0.99)
  const float dLg = (on && __fmul_rn(q1.y, G) <= kAlphaClamp) ? dLda : 0.f;
  acc[5] = fmaf(dLg, G, acc[5]);
  const float dp = dLg * alpha;  // dL/dpower
  acc[0] = fmaf(dp, fmaf(q0.w, dy, cA2dx), acc[0]);       // d p2 / d mu_x
  acc[1] = fmaf(dp, fmaf(2.f * q1.x, dy, cBdx), acc[1]);  // d p2 / d mu_y
  acc[2] = fmaf(dp, dx2, acc[2]);
  acc[3] = fmaf(dp, dx * dy, acc[3]);
  acc[4] = fmaf(dp, dy * dy, acc[4]);
  return on;
}

// One forward (pixel, Gaussian) pair, branch-free.  bit = this pixel's bit in
// `done`; idx = 1 + the pair's list position.
__device__ __forceinline__ bool fwd_pair(const float4& q1, float blue, float a0, float a1, float dy, uint32_t bit,
                                         uint32_t idx, uint32_t& done, float& T, float (&C)[3], uint32_t& last) {
  const float p2 = splat_p2(q1.x, a1, a0, dy);
  float G;
  const float alpha = splat_alpha2(q1.y, p2, G);
  const bool ok = !(done & bit) && !(p2 > 0.f) && !(alpha < kAlphaSkip);
  const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
  const bool stop = ok && Tn < kTStop;
  done |= stop ? bit : 0u;
  const bool acc = ok && !stop;
  const float wgt = acc ? alpha * T : 0.f;
  C[0] = fmaf(q1.z, wgt, C[0]);
  C[1] = fmaf(q1.w, wgt, C[1]);
  C[2] = fmaf(blue, wgt, C[2]);
  T = acc ? Tn : T;
  last = acc ? idx : last;
  return acc;
}

// ---------------------------------------------------------------- pixel pairs
//
// With two or more pixels per thread, the pixels of a pair (rows k and k + 1
// of one column: same dx, different dy) go through the packed FP32x2
// instructions of sm_100-class GPUs, one instruction for both.  Each element
// is rounded exactly like the scalar operation it replaces (dy = mu_y - y is
// computed as mu_y + (-y), which IEEE defines identically), so every skip and
// stop decision equals the one-pixel variant's.

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// Forward of one pixel pair (bits bitx, bitx << 1 of `done`).
__device__ __forceinline__ bool fwd_pair2(const float2& cC, const float2& a1, const float2& a0, const float2& op,
                                          const float2& r, const float2& g, const float2& b, float2 dy,
                                          uint32_t bitx, uint32_t idx, uint32_t& done, float2& T, float2 (&C)[3],
                                          uint32_t& lastx, uint32_t& lasty) {
  const float2 p2 = __ffma2_rn(__ffma2_rn(cC, dy, a1), dy, a0);
  const float2 raw = __fmul2_rn(op, make_float2(ex2_approx(p2.x), ex2_approx(p2.y)));
  const float ax = fminf(kAlphaClamp, raw.x), ay = fminf(kAlphaClamp, raw.y);
  const uint32_t bity = bitx << 1;
  const bool okx = !(done & bitx) && !(p2.x > 0.f) && !(ax < kAlphaSkip);
  const bool oky = !(done & bity) && !(p2.y > 0.f) && !(ay < kAlphaSkip);
  const float2 Tn = __fmul2_rn(T, __fadd2_rn(bc2(1.f), make_float2(-ax, -ay)));
  const bool stx = okx && Tn.x < kTStop, sty = oky && Tn.y < kTStop;
  done |= (stx ? bitx : 0u) | (sty ? bity : 0u);
  const bool accx = okx && !stx, accy = oky && !sty;
  const float2 aT = __fmul2_rn(make_float2(ax, ay), T);
  const float2 w = make_float2(accx ? aT.x : 0.f, accy ? aT.y : 0.f);
  C[0] = __ffma2_rn(r, w, C[0]);
  C[1] = __ffma2_rn(g, w, C[1]);
  C[2] = __ffma2_rn(b, w, C[2]);
  T = make_float2(accx ? Tn.x : T.x, accy ? Tn.y : T.y);
  lastx = accx ? idx : lastx;
  lasty = accy ? idx : lasty;
  return accx || accy;
}

// Backward of one pixel pair.  Per (thread, Gaussian) it accumulates the
// colour and opacity gradients and three moments of dL/dp2 over the pixels
// (S0 = sum dp, S1 = sum dp dy, S2 = sum dp dy^2), from which the mean and
// conic gradients follow once per Gaussian.  Returns whether a pixel of the
// pair contributed.
__device__ __forceinline__ bool bwd_pair2(bool livex, bool livey, const float2& cC, const float2& a1,
                                          const float2& a0, const float2& op, const float2& r, const float2& g,
                                          const float2& b, float2 dy, float2& T, float2& dCS, const float2 (&dC)[3],
                                          const float2& bgd, float2 (&racc)[3], float2& oacc, float2& S0,
                                          float2& S1, float2& S2) {
  const float2 p2 = __ffma2_rn(__ffma2_rn(cC, dy, a1), dy, a0);
  const float2 G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
  const float2 raw = __fmul2_rn(op, G);
  const float ax = fminf(kAlphaClamp, raw.x), ay = fminf(kAlphaClamp, raw.y);
  const bool onx = livex && !(p2.x > 0.f) && !(ax < kAlphaSkip);
  const bool ony = livey && !(p2.y > 0.f) && !(ay < kAlphaSkip);
  const float2 ae = make_float2(onx ? ax : 0.f, ony ? ay : 0.f);
  const float2 om = __fadd2_rn(bc2(1.f), make_float2(-ae.x, -ae.y));
  // 1 - ae is in [0.01, 1]: the approximate reciprocal (relative error
  // below 2^-22) keeps the recovered T within FP32 rounding of the division
  const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
  const float2 Ti = __fmul2_rn(T, inv);
  const float2 w = __fmul2_rn(ae, Ti);
  const float2 dcr = __ffma2_rn(dC[2], b, __ffma2_rn(dC[1], g, __fmul2_rn(dC[0], r)));
  // dL/dalpha = T_i (dC . rgb) - (bg T_final + S) . dC / (1 - alpha)
  const float2 dLda = __ffma2_rn(Ti, dcr, __fmul2_rn(make_float2(-inv.x, -inv.y), __fadd2_rn(bgd, dCS)));
  racc[0] = __ffma2_rn(dC[0], w, racc[0]);
  racc[1] = __ffma2_rn(dC[1], w, racc[1]);
  racc[2] = __ffma2_rn(dC[2], w, racc[2]);
  dCS = __ffma2_rn(w, dcr, dCS);
  T = Ti;
  // zero through a clamped alpha (opacity G > 0.99)
  const float2 dLg = make_float2((onx && raw.x <= kAlphaClamp) ? dLda.x : 0.f,
                                 (ony && raw.y <= kAlphaClamp) ? dLda.y : 0.f);
  oacc = __ffma2_rn(dLg, G, oacc);
  const float2 dp = __fmul2_rn(dLg, make_float2(ax, ay));  // dL/dpower
  S0 = __fadd2_rn(S0, dp);
  const float2 t = __fmul2_rn(dp, dy);
  S1 = __fadd2_rn(S1, t);
  S2 = __ffma2_rn(t, dy, S2);
  return onx || ony;
}

// ---------------------------------------------------------------- launch shapes
//
// PPT = pixels per thread.  A block holds TPB tiles; a warp owns a WR x HR
// pixel rectangle of its tile (lane l: column l % CW, rows (l / CW) * PPT + k)
// and walks the tile's list on its own: it stages 32 records at a time into
// its own shared slots and never waits for the other warps of the block.
template <int PPT>
struct Shape;
template <>
struct Shape<1> {  // 8 warps per tile, 8 x 4 pixels each
  static constexpr int NW = 8, TPB = 1, CW = 8;
};
template <>
struct Shape<2> {  // 4 warps per tile, 8 x 8 pixels each
  static constexpr int NW = 4, TPB = 1, CW = 8;
};
template <>
struct Shape<4> {  // 2 warps per tile, 8 x 16 pixels each
  static constexpr int NW = 2, TPB = 1, CW = 8;
};
template <>
struct Shape<8> {  // 1 warp per tile, 4 tiles per block
  static constexpr int NW = 1, TPB = 4, CW = 16;
};

// Lane groups: the warp's lanes form NG = 32 / GW groups, each owning a
// GCW x GRH sub-rectangle of the warp's pixels and walking only the
// Gaussians whose box reaches it (the warp iterates max over groups; a lane
// whose group has run out takes no-op steps).  With 2 pixels per thread
// both kernels use 8 groups of 2 x 4 pixels (one contribution cell each).
template <int PPT>
struct LaneGroups {
  static constexpr int FWD = PPT == 2 ? 4 : 32;
  static constexpr int BWD = PPT == 2 ? 4 : 32;
};

template <int PPT, int GWv = 32>
struct Geo {
  static constexpr int NW = Shape<PPT>::NW, TPB = Shape<PPT>::TPB, CW = Shape<PPT>::CW;
  static constexpr int THREADS = 32 * NW * TPB;
  static constexpr int RW = CW, RH = (32 / CW) * PPT;  // warp rectangle
  // lane groups: NG groups of GW lanes, each a GCW x GRH pixel rectangle
  static constexpr int GW = GWv, NG = 32 / GW;
  static constexpr int GCW = GW >= 16 ? CW : GW / 2, GRH = (GW / GCW) * PPT, NGX = RW / GCW;
  int64_t bin;
  int v, px, py0, grp;
  float wx0, wx1, wy0, wy1;
  // rectangle of lane group g
  __device__ __forceinline__ void group_rect(int g, float& x0, float& x1, float& y0, float& y1) const {
    x0 = wx0 + (float)((g % NGX) * GCW);
    x1 = x0 + (float)(GCW - 1);
    y0 = wy0 + (float)((g / NGX) * GRH);
    y1 = y0 + (float)(GRH - 1);
  }
  __device__ bool init(const RasterArgs& a, int64_t bins, int warp, int lane) {
    const int tile_in_block = warp / NW, sub = warp % NW;
    bin = (int64_t)blockIdx.x * TPB + tile_in_block;
    if (bin >= bins) return false;
    if (a.tile_order) bin = a.tile_order[bin];
    v = view_of_bin(a.views, a.B, (int)bin);
    const ViewRec& V = a.views[v];
    const int tile = (int)bin - V.tile_offset;
    const int tx = tile % V.gw, ty = tile / V.gw;
    const int ox = (sub % (kTile / RW)) * RW, oy = (sub / (kTile / RW)) * RH;
    grp = lane / GW;
    const int gl = lane % GW;
    px = tx * kTile + ox + (grp % NGX) * GCW + (gl % GCW);
    py0 = ty * kTile + oy + (grp / NGX) * GRH + (gl / GCW) * PPT;
    wx0 = (float)(tx * kTile + ox);
    wx1 = wx0 + (float)(RW - 1);
    wy0 = (float)(ty * kTile + oy);
    wy1 = wy0 + (float)(RH - 1);
    return true;
  }
};

// Contribution cells: a tile is 8 x 4 cells of 2 x 4 pixels, cell
// c = x / 2 + 8 (y / 4) in tile coordinates.  For every batch of 32 list
// entries (entries 32 k .. 32 k + 31 of the tile's list) the forward stores,
// per cell, the mask of the entries that contributed to a pixel of the cell:
// word cells_offset(start, bin) + 32 k + c, start = the tile's first sorted
// instance.  The offset pads every tile's region to whole batches (a buffer
// of instances + 32 bins words), so tiles never share a word, and each cell
// belongs to one warp of the forward, which writes every batch of its
// tile's list (zero after its pixels stopped).  The backward walks an entry
// only in the lane groups whose cell it contributed to.
__device__ __forceinline__ int64_t cells_offset(uint32_t start, int64_t bin) { return (int64_t)start + 32 * bin; }

__device__ __forceinline__ int cell_index(int px, int py) {
  return ((px & (kTile - 1)) >> 1) + 8 * ((py & (kTile - 1)) >> 2);
}
template <int PPT>
__global__ void __launch_bounds__(Geo<PPT>::THREADS) raster_fwd_kernel(RasterArgs a, int64_t bins) {
  using G = Geo<PPT, LaneGroups<PPT>::FWD>;
  constexpr int NWB = G::NW * G::TPB;  // warps per block
  constexpr int NP = PPT / 2;          // pixel pairs per thread
  __shared__ float4 s0[NWB][32], s1[NWB][32], s2[NWB][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  G geo;
  if (!geo.init(a, bins, w, lane)) {
    return;  // a warp past the last tile (one-warp-per-tile shape): no pixels
  }
  const int v = geo.v, px = geo.px, py0 = geo.py0;
  const ViewRec& V = a.views[v];
  const uint2 rg = a.ranges[geo.bin];
  const int n = (int)(rg.y - rg.x);
  const uint32_t* __restrict__ vals = *a.vals;

  // PPT == 1: scalar state; otherwise pixel pairs (pixel k = pair k / 2,
  // element k % 2)
  float T[PPT], C[PPT][3];
  float2 T2[NP > 0 ? NP : 1], C2[NP > 0 ? NP : 1][3], nfy[NP > 0 ? NP : 1];
  uint32_t last[PPT];
  uint32_t done = 0;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    T[k] = 1.f;
    C[k][0] = C[k][1] = C[k][2] = 0.f;
    last[k] = 0;
    if (!(px < V.W && py0 + k < V.H)) done |= 1u << k;
  }
#pragma unroll
  for (int j = 0; j < NP; j++) {
    T2[j] = bc2(1.f);
    C2[j][0] = C2[j][1] = C2[j][2] = bc2(0.f);
    nfy[j] = make_float2(-((float)py0 + (float)(2 * j)), -((float)py0 + (float)(2 * j + 1)));
  }
  const uint32_t all_done = (1u << PPT) - 1u;
  const float fpx = (float)px, fpy = (float)py0;
  // contribution cells: a lane's pixels lie in NSL cells (one per 4 rows;
  // py0 is even, and a multiple of 4 with 4+ pixels per thread); per batch
  // a lane keeps, per cell, the mask of the entries it contributed to
  constexpr int NSL = PPT >= 4 ? PPT / 4 : 1;
  // the lanes of a cell hold its mask after an OR over the lane bits that
  // select the column within the pair (bit 0) and, with fewer than 4 pixels
  // per thread, the row block within the cell (lane bits from GCW up); the
  // lane whose bits there are 0 stores it (each cell belongs to one warp)
  constexpr int RB = PPT < 4 ? 4 / PPT : 1;  // lane rows per cell
  const bool owner = (lane & 1) == 0 && ((lane / G::GCW) % RB) == 0;
  uint32_t* const cell_base = a.cells ? a.cells + cells_offset(rg.x, geo.bin) : nullptr;
  int b0 = 0;
  // software pipeline over the batches: the record of batch k + 1 and the
  // index of batch k + 2 are loaded while batch k is walked
  uint32_t g_next = lane < n ? vals[rg.x + lane] : 0u;
  uint32_t g_after = 32 + lane < n ? vals[rg.x + 32 + lane] : 0u;
  float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0, p2 = p0;
  if (lane < n) stage_one(a, v, g_next, p0, p1, p2);
  for (; b0 < n; b0 += 32) {
    if (__all_sync(0xffffffffu, done == all_done)) break;
    const int i = b0 + lane;
    bool hit = false;
    __syncwarp();
    uint32_t cm[NSL];
#pragma unroll
    for (int sl = 0; sl < NSL; sl++) cm[sl] = 0u;
    uint32_t gbits = 0;
    if (i < n) {
      const float4 r0 = p0, r1 = p1, r2 = p2;
      s0[w][lane] = r0;
      s1[w][lane] = r1;
      s2[w][lane] = r2;
      if constexpr (G::NG > 1) gbits = box_group_bits(r0, r2, geo);
      else hit = ellipse_hits(r0, r1, r2, geo.wx0, geo.wx1, geo.wy0, geo.wy1);
    }
    {
      const int i1 = i + 32, i2 = i + 64;
      if (i1 < n) stage_one(a, v, g_after, p0, p1, p2);
      g_after = i2 < n ? vals[rg.x + i2] : 0u;
    }
    // each lane culls its own record; the warp (each lane group) walks the
    // survivors in order
    uint32_t mask = __ballot_sync(0xffffffffu, hit);
    int iters = 32;
    if constexpr (G::NG > 1) {
#pragma unroll
      for (int g = 0; g < G::NG; g++) {
        const uint32_t m = __ballot_sync(0xffffffffu, (gbits >> g) & 1u);
        mask = g == geo.grp ? m : mask;
      }
      // a group whose pixels have all stopped walks nothing more
      const uint32_t fin = __ballot_sync(0xffffffffu, done == all_done);
      const uint32_t gm = G::GW == 32 ? 0xffffffffu : ((1u << (G::GW % 32)) - 1u) << (geo.grp * G::GW);
      if ((fin & gm) == gm) mask = 0u;
      iters = (int)__reduce_max_sync(0xffffffffu, (uint32_t)__popc(mask));
    }
    __syncwarp();
    for (int it = 0; G::NG > 1 ? it < iters : mask != 0u; it++) {
      const bool act = mask != 0u;
      // (an idle group evaluates slot 0, which every batch stages: b0 < n)
      const int j = act ? __ffs(mask) - 1 : 0;
      mask &= mask - 1u;
      const float4 q0 = s0[w][j];
      const float4 q2 = s2[w][j];
      const float4 q1 = s1[w][j];
      const float dx = __fsub_rn(q0.x, fpx);
      const float a0 = __fmul_rn(q0.z, __fmul_rn(dx, dx));
      const float a1 = __fmul_rn(q0.w, dx);
      const uint32_t idx = (uint32_t)(b0 + j + 1);
      const uint32_t jbit = 1u << j;
      if constexpr (NP == 0) {
#pragma unroll
        for (int k = 0; k < PPT; k++)
          cm[0] |= fwd_pair(q1, q2.x, a0, a1, __fsub_rn(q0.y, fpy + (float)k), 1u << k, idx, done, T[k], C[k],
                            last[k]) ? jbit : 0u;
      } else {
        const float2 cC = bc2(q1.x), A1 = bc2(a1), A0 = bc2(a0), op = bc2(q1.y);
        const float2 r = bc2(q1.z), g = bc2(q1.w), b = bc2(q2.x), qy = bc2(q0.y);
        // a lane whose group has no survivor left changes nothing
        uint32_t dn = act ? done : all_done;
#pragma unroll
        for (int jp = 0; jp < NP; jp++)
          cm[jp / 2 < NSL ? jp / 2 : 0] |= fwd_pair2(cC, A1, A0, op, r, g, b, __fadd2_rn(qy, nfy[jp]), 1u << (2 * jp),
                                                   idx, dn, T2[jp], C2[jp], last[2 * jp], last[2 * jp + 1]) ? jbit : 0u;
        done = act ? dn : done;
      }
    }
    // the batch's contribution masks: per cell, the OR of its lanes' entry masks
    if (cell_base) {
#pragma unroll
      for (int sl = 0; sl < NSL; sl++) {
        uint32_t e = cm[sl] | __shfl_xor_sync(0xffffffffu, cm[sl], 1);
#pragma unroll
        for (int x = G::GCW; x < G::GCW * RB; x <<= 1) e |= __shfl_xor_sync(0xffffffffu, e, x);
        if (owner) cell_base[b0 + cell_index(px, py0 + 4 * sl)] = e;
      }
    }
  }
  // batches after the warp's pixels all stopped: nothing contributed
  if (cell_base && owner)
    for (; b0 < n; b0 += 32)
#pragma unroll
      for (int sl = 0; sl < NSL; sl++) cell_base[b0 + cell_index(px, py0 + 4 * sl)] = 0u;
  if constexpr (NP > 0) {
#pragma unroll
    for (int jp = 0; jp < NP; jp++) {
      T[2 * jp] = T2[jp].x;
      T[2 * jp + 1] = T2[jp].y;
#pragma unroll
      for (int c = 0; c < 3; c++) {
        C[2 * jp][c] = C2[jp][c].x;
        C[2 * jp + 1][c] = C2[jp][c].y;
      }
    }
  }
  const int64_t plane = (int64_t)V.W * V.H;
  float* img = a.image ? a.image + 3 * V.pix_offset : nullptr;
  const float* tgt = a.target_slot ? *a.target_slot : a.target;
  const bool l1 = tgt != nullptr;
  // the targets are loaded before any store (the stores could alias them,
  // which would serialise each load behind the stores before it)
  float tv[PPT][3];
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int py = py0 + k;
    const bool in = l1 && px < V.W && py < V.H;
    const int64_t p = (int64_t)py * V.W + px;
#pragma unroll
    for (int ch = 0; ch < 3; ch++) tv[k][ch] = in ? __ldg(tgt + 3 * V.pix_offset + ch * plane + p) : 0.f;
  }
  float l1sum = 0.f;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int py = py0 + k;
    if (px >= V.W || py >= V.H) continue;
    const int64_t p = (int64_t)py * V.W + px;
    const float c0 = fmaf(T[k], V.bg[0], C[k][0]);
    const float c1 = fmaf(T[k], V.bg[1], C[k][1]);
    const float c2 = fmaf(T[k], V.bg[2], C[k][2]);
    if (img) {
      img[p] = c0;
      img[plane + p] = c1;
      img[2 * plane + p] = c2;
    }
    a.tfinal[V.pix_offset + p] = T[k];
    a.nlast[V.pix_offset + p] = last[k];
    if (l1) {
      // L1 loss mean |C - target| and its gradient sign(C - target) / count
      float* gd = a.l1_grad + 3 * V.pix_offset;
      const float cc[3] = {c0, c1, c2};
#pragma unroll
      for (int ch = 0; ch < 3; ch++) {
        const float d = cc[ch] - tv[k][ch];
        l1sum += fabsf(d);
        gd[ch * plane + p] = d > 0.f ? a.inv_count : (d < 0.f ? -a.inv_count : 0.f);
      }
    }
  }
  if (l1) {
    // one partial sum per warp (fixed order: deterministic)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l1sum += __shfl_down_sync(0xffffffffu, l1sum, off);
    // indexed by tile, so the loss does not depend on the tile order
    if (lane == 0) a.l1_partial[geo.bin * G::NW + (w % G::NW)] = l1sum;
  }
}

template <int PPT>
__global__ void __launch_bounds__(Geo<PPT>::THREADS, PPT == 2 ? 8 : 1) raster_bwd_kernel(RasterArgs a, int64_t bins) {
  using G = Geo<PPT, LaneGroups<PPT>::BWD>;
  constexpr int NWB = G::NW * G::TPB;
  constexpr int NP = PPT / 2;  // pixel pairs per thread (0: the scalar one-pixel path)
  constexpr int NS = NP > 0 ? NP : 1;
  __shared__ float4 s0[NWB][32], s1[NWB][32], s2[NWB][32];
  __shared__ uint32_t sg[NWB][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  G geo;
  if (!geo.init(a, bins, w, lane)) return;
  const int v = geo.v, px = geo.px, py0 = geo.py0;
  const ViewRec& V = a.views[v];
  const uint2 rg = a.ranges[geo.bin];
  const uint32_t* __restrict__ vals = *a.vals;
  const int64_t plane = (int64_t)V.W * V.H;
  const float* dimg = a.dimage + 3 * V.pix_offset;

  // per pixel: T (running, from T_final backwards), dL/dC, sum_c dC_c S_c
  // (S = colour behind), T_final * sum_c dC_c bg_c, and n_last
  float T[PPT], dC[PPT][3], dCS[PPT], bgd[PPT];
  uint32_t nl[PPT];
  uint32_t mymax = 0;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int py = py0 + k;
    const bool in = px < V.W && py < V.H;
    const int64_t p = (int64_t)py * V.W + px;
    T[k] = in ? a.tfinal[V.pix_offset + p] : 1.f;
    nl[k] = in ? a.nlast[V.pix_offset + p] : 0u;
#pragma unroll
    for (int c = 0; c < 3; c++) dC[k][c] = in ? dimg[c * plane + p] : 0.f;
    dCS[k] = 0.f;
    bgd[k] = T[k] * (dC[k][0] * V.bg[0] + dC[k][1] * V.bg[1] + dC[k][2] * V.bg[2]);
    mymax = max(mymax, nl[k]);
  }
  // the same state as pixel pairs
  float2 T2[NS], dC2[NS][3], dCS2[NS], bgd2[NS], nfy[NS];
#pragma unroll
  for (int j = 0; j < NP; j++) {
    T2[j] = make_float2(T[2 * j], T[2 * j + 1]);
#pragma unroll
    for (int c = 0; c < 3; c++) dC2[j][c] = make_float2(dC[2 * j][c], dC[2 * j + 1][c]);
    dCS2[j] = bc2(0.f);
    bgd2[j] = make_float2(bgd[2 * j], bgd[2 * j + 1]);
    nfy[j] = make_float2(-((float)py0 + (float)(2 * j)), -((float)py0 + (float)(2 * j + 1)));
  }
  // this warp only walks the entries before its pixels' last contributors
  const int total = (int)__reduce_max_sync(0xffffffffu, mymax);
  const float fpx = (float)px, fpy = (float)py0;
  // contribution masks of the forward (batches of 32 entries from the
  // front of the list, one mask per cell): lane k < NCX NCY loads the mask
  // of the warp's k-th cell; the warp walks the union, each lane group the
  // mask of its own cell
  constexpr int NCX = G::RW / 2, NCY = G::RH / 4;
  static_assert(G::NG == 1 || (G::GCW == 2 && G::GRH == 4 && G::NGX == NCX), "one contribution cell per lane group");
  const int c00 = (((int)geo.wx0 & (kTile - 1)) >> 1) + 8 * (((int)geo.wy0 & (kTile - 1)) >> 2);
  const uint32_t* __restrict__ cell_base =
      a.cells + cells_offset(rg.x, geo.bin) + c00 + lane % NCX + 8 * (lane / NCX);
  // the cell masks of the next batch are loaded while a batch is walked
  const int btop = ((total - 1) >> 5) << 5;
  uint32_t cm_next = (total > 0 && lane < NCX * NCY) ? cell_base[btop] : 0u;
  for (int bstart = btop; bstart >= 0 && total > 0; bstart -= 32) {
    const int i = bstart + lane;
    // entries at or past the warp's last contributor change nothing
    const int nb = min(32, total - bstart);
    const uint32_t lim = nb >= 32 ? 0xffffffffu : (1u << nb) - 1u;
    const uint32_t cm = cm_next & lim;
    cm_next = (bstart >= 32 && lane < NCX * NCY) ? cell_base[bstart - 32] : 0u;
    const uint32_t any = __reduce_or_sync(0xffffffffu, cm);
    // a batch where nothing contributed to the warp's pixels is skipped
    // without loading its records
    if (any == 0u) continue;
    __syncwarp();
    if ((any >> lane) & 1u) {
      const uint32_t ng = vals[rg.x + i];
      float4 n0, n1, n2;
      stage_one(a, v, ng, n0, n1, n2);
      s0[w][lane] = n0;
      s1[w][lane] = n1;
      s2[w][lane] = n2;
      sg[w][lane] = ng;
    }
    // group g's cell is the warp's cell g (groups of 2 x 4 pixels)
    uint32_t mask = G::NG > 1 ? __shfl_sync(0xffffffffu, cm, geo.grp) : any;
    int iters = 32;
    if constexpr (G::NG > 1) iters = (int)__reduce_max_sync(0xffffffffu, (uint32_t)__popc(mask));
    // a group that has run out of entries evaluates a staged one with no
    // effect: a slot this batch did not stage holds stale shared memory,
    // whose infinities would turn the zero-weighted updates into NaN
    const int j_idle = 31 - __clz(any);
    __syncwarp();
    for (int it = 0; G::NG > 1 ? it < iters : mask != 0u; it++) {  // back to front
      const bool act = mask != 0u;
      const int j = act ? 31 - __clz(mask) : j_idle;
      mask = act ? mask ^ (1u << j) : 0u;
      const float4 q0 = s0[w][j];
      const float4 q2 = s2[w][j];
      const float4 q1 = s1[w][j];
      const uint32_t idx = (uint32_t)(bstart + j);
      const float dx = __fsub_rn(q0.x, fpx);
      const float dx2 = __fmul_rn(dx, dx);
      const float a0 = __fmul_rn(q0.z, dx2);
      const float a1 = __fmul_rn(q0.w, dx);
      const float cA2dx = 2.f * q0.z * dx;
      const float cBdx = q0.w * dx;
      float acc[16];
#pragma unroll
      for (int q = 0; q < 16; q++) acc[q] = 0.f;
      bool any = false;
      if constexpr (NP == 0) {
        const float rgb[3] = {q1.z, q1.w, q2.x};
#pragma unroll
        for (int k = 0; k < PPT; k++)
          any |= bwd_pair(act && idx < nl[k], q0, q1, rgb, a0, a1, __fsub_rn(q0.y, fpy + (float)k), dx, dx2, cA2dx, cBdx,
                          T[k], dCS[k], dC[k], bgd[k], acc);
      } else {
        const float2 cC = bc2(q1.x), A1 = bc2(a1), A0 = bc2(a0), op = bc2(q1.y);
        const float2 r = bc2(q1.z), g = bc2(q1.w), b = bc2(q2.x), qy = bc2(q0.y);
        float2 racc[3] = {bc2(0.f), bc2(0.f), bc2(0.f)}, oacc = bc2(0.f);
        float2 S0 = bc2(0.f), S1 = bc2(0.f), S2 = bc2(0.f);
#pragma unroll
        for (int jp = 0; jp < NP; jp++)
          any |= bwd_pair2(act && idx < nl[2 * jp], act && idx < nl[2 * jp + 1], cC, A1, A0, op, r, g, b,
                           __fadd2_rn(qy, nfy[jp]), T2[jp], dCS2[jp], dC2[jp], bgd2[jp], racc, oacc, S0, S1, S2);
        // mean and conic gradients of p2 from the moments of dL/dp2
        const float m0 = S0.x + S0.y, m1 = S1.x + S1.y;
        acc[0] = fmaf(q0.w, m1, cA2dx * m0);        // sum dp (cB dy + 2 cA dx)
        acc[1] = fmaf(2.f * q1.x, m1, cBdx * m0);   // sum dp (2 cC dy + cB dx)
        acc[2] = dx2 * m0;
        acc[3] = dx * m1;
        acc[4] = S2.x + S2.y;
        acc[5] = oacc.x + oacc.y;
#pragma unroll
        for (int c = 0; c < 3; c++) acc[6 + c] = racc[c].x + racc[c].y;
      }
      const uint32_t contrib = __ballot_sync(0xffffffffu, any);
      if (contrib)
        push_grad_group<G::GW>(a.g2d, (int64_t)a.B * a.stride, (int64_t)v * a.stride + sg[w][j], acc, lane, contrib,
                               a.direct_max);
    }
  }
}

template <int PPT>
void launch_shape(bool fwd, const RasterArgs& a, int64_t bins, cudaStream_t s) {
  using G = Geo<PPT>;
  const unsigned blocks = (unsigned)((bins + G::TPB - 1) / G::TPB);
  if (fwd) raster_fwd_kernel<PPT><<<blocks, G::THREADS, 0, s>>>(a, bins);
  else raster_bwd_kernel<PPT><<<blocks, G::THREADS, 0, s>>>(a, bins);
}

int64_t raster_fwd_warps(int64_t bins, int ppt) {
  // L1 partial sums of a fused forward: one per warp of each tile
  switch (ppt) {
    case 1: return bins * Geo<1>::NW;
    case 4: return bins * Geo<4>::NW;
    case 8: return bins * Geo<8>::NW;
    default: return bins * Geo<2>::NW;
  }
}

// Sum of the partials in a fixed order: 256 blocks each add a strided
// subset (FP64, a handful of terms per thread) and a tree inside the block;
// one block adds the 256 block sums.  The loss is deterministic.
constexpr int kL1FinishBlocks = 256;

__global__ void __launch_bounds__(256) l1_partials_kernel(const float* __restrict__ partial, int64_t nparts,
                                                          double* __restrict__ block_sums) {
  __shared__ double red[8];
  double t = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nparts; i += (int64_t)gridDim.x * blockDim.x)
    t += partial[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < 8; w++) u += red[w];
    block_sums[blockIdx.x] = u;
  }
}

__global__ void __launch_bounds__(256) l1_finish_tree_kernel(const double* __restrict__ block_sums, double inv_count,
                                                             float* loss) {
  __shared__ double red[8];
  double t = threadIdx.x < kL1FinishBlocks ? block_sums[threadIdx.x] : 0.0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < 8; w++) u += red[w];
    *loss = (float)(u * inv_count);
  }
}

int64_t l1_finish_scratch_bytes() { return kL1FinishBlocks * sizeof(double); }

void launch_l1_finish(const float* partial, int64_t nparts, double* scratch, double inv_count, float* loss,
                      cudaStream_t s) {
  l1_partials_kernel<<<kL1FinishBlocks, 256, 0, s>>>(partial, nparts, scratch);
  l1_finish_tree_kernel<<<1, 256, 0, s>>>(scratch, inv_count, loss);
}

// Work counters of the last forward pass (inspection, outside the training
// step): per pixel, the list entries up to and including its last
// contributor (n_last: what the backward walks, and a lower bound of what
// the forward walks) and, among them, the pairs that pass the power <= 0
// and alpha >= 1/255 tests (the contributing pairs), evaluated with the
// compositing kernels' own instruction sequence.  One block per tile, one
// thread per pixel; out[0] += entries, out[1] += contributing pairs.
__global__ void __launch_bounds__(256) pair_stats_kernel(RasterArgs a, unsigned long long* out) {
  const int bin = (int)blockIdx.x;
  const int v = view_of_bin(a.views, a.B, bin);
  const ViewRec& V = a.views[v];
  const int tile = bin - V.tile_offset;
  const int px = (tile % V.gw) * kTile + (int)(threadIdx.x & 15);
  const int py = (tile / V.gw) * kTile + (int)(threadIdx.x >> 4);
  const uint2 rg = a.ranges[bin];
  const uint32_t* __restrict__ vals = *a.vals;
  uint32_t nl = 0;
  if (px < V.W && py < V.H) nl = a.nlast[V.pix_offset + (int64_t)py * V.W + px];
  nl = min(nl, rg.y - rg.x);
  unsigned long long entries = nl, contrib = 0;
  const float fpx = (float)px, fpy = (float)py;
  for (uint32_t i = 0; i < nl; i++) {
    float4 r0, r1, r2;
    stage_one(a, v, vals[rg.x + i], r0, r1, r2);
    const float dx = __fsub_rn(r0.x, fpx);
    const float a0 = __fmul_rn(r0.z, __fmul_rn(dx, dx));
    const float a1 = __fmul_rn(r0.w, dx);
    const float p2 = splat_p2(r1.x, a1, a0, __fsub_rn(r0.y, fpy));
    float G;
    const float alpha = splat_alpha2(r1.y, p2, G);
    contrib += (!(p2 > 0.f) && !(alpha < kAlphaSkip)) ? 1ull : 0ull;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    entries += __shfl_down_sync(0xffffffffu, entries, off);
    contrib += __shfl_down_sync(0xffffffffu, contrib, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, entries);
    atomicAdd(out + 1, contrib);
  }
}

void launch_pair_stats(const RasterArgs& a, int64_t bins, unsigned long long* out, cudaStream_t s) {
  if (bins == 0) return;
  pair_stats_kernel<<<(unsigned)bins, 256, 0, s>>>(a, out);
}

void launch_raster_fwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s) {
  if (bins == 0) return;
  switch (ppt) {
    case 1: launch_shape<1>(true, a, bins, s); break;
    case 4: launch_shape<4>(true, a, bins, s); break;
    case 8: launch_shape<8>(true, a, bins, s); break;
    default: launch_shape<2>(true, a, bins, s); break;
  }
}

void launch_raster_bwd(const RasterArgs& a, int64_t bins, int ppt, cudaStream_t s) {
  if (bins == 0) return;
  switch (ppt) {
    case 1: launch_shape<1>(false, a, bins, s); break;
    case 4: launch_shape<4>(false, a, bins, s); break;
    case 8: launch_shape<8>(false, a, bins, s); break;
    default: launch_shape<2>(false, a, bins, s); break;
  }
}

}  // namespace gs
