// fd_kernels_plain.cuh -- plain stencil kernels, setup kernels, sparse kernels.
//
// The plain stencil kernel computes one grid point per thread and reads its
// 2·D·R neighbours straight from global memory (L1/L2 serve the re-reads).
// It is the simple design the pipelined kernel is measured against, and the
// path for 2-D grids.
#pragma once

#include "fd_common.cuh"

namespace fdk {

// ---------------------------------------------------------------------------
// One time step, plain.  Block (32, 8): x along lanes, y along warps; grid.z = z.
// L u = Σ_axes Σ_k w_k/h² ((u_{+k} + u_{-k}) - 2u)  (the centre weight is implied)
//   diffusion: un = u + (ν dt L) u on interior nodes (coefficients carry ν dt)
//   acoustic : un = A·(L u) + (1 + C)·u − C·un   (un holds u^{n-1} on entry)
// with A = dt²/(m+σ), C = (m−σ)/(m+σ): the leapfrog update solved for u^{n+1}.
// ---------------------------------------------------------------------------
// L u at one point from its centre value and neighbour reads nb(axis, ±k): the
// operation sequence every plain-order kernel shares (so they agree bitwise).
// Difference form: the weights of every pair sum to zero exactly, so the FP32
// operator annihilates constants (no drift from rounded weights).  One FMA chain
// runs over the y offsets, then continues over x (then z): a kernel that streams
// rows takes the y part from a register queue and the x part from the staged row.
// ISO2 (2-D, equal spacing): one weight per offset multiplies the sum of the four
// neighbours minus 4u, ((u_{y+k} + u_{y-k}) + (u_{x+k} + u_{x-k})) - 4u: five
// operations an offset instead of six, still exact on constants (2c + 2c = 4c and
// 4u are exact), as the 3-D pipelined kernels do for equal spacing.
template <int R, bool THREE_D, typename NB, bool ISO2 = false>
__device__ __forceinline__ float plain_lap(float uc, const Coef &c, NB nb) {
  if constexpr (ISO2 && !THREE_D) {
    const float nuc4 = -4.f * uc;
    float lap = 0.f;
#pragma unroll
    for (int k = 1; k <= R; ++k)
      lap = fmaf(c.w[2][k], ((nb(1, k) + nb(1, -k)) + (nb(2, k) + nb(2, -k))) + nuc4, lap);
    return lap;
  }
  const float uc2 = uc + uc;
  float lap = 0.f;
#pragma unroll
  for (int k = 1; k <= R; ++k) lap = fmaf(c.w[1][k], (nb(1, k) + nb(1, -k)) - uc2, lap);
#pragma unroll
  for (int k = 1; k <= R; ++k) lap = fmaf(c.w[2][k], (nb(2, k) + nb(2, -k)) - uc2, lap);
  if (THREE_D) {
#pragma unroll
    for (int k = 1; k <= R; ++k) lap = fmaf(c.w[0][k], (nb(0, k) + nb(0, -k)) - uc2, lap);
  }
  return lap;
}

// The acoustic update from the Laplacian: A·lap + (1 + C)·u − C·u^{n−1}.
__device__ __forceinline__ float leapfrog(float a, float cc, float uc, float prev, float lap) {
  return fmaf(a, lap, fmaf(1.f + cc, uc, -cc * prev));
}

template <int R, int EQ, bool THREE_D, bool ISO2 = false>
__device__ __forceinline__ void plain_point(const float *__restrict__ u, float *un,
                                            const float *__restrict__ A,
                                            const float *__restrict__ C, const Geom &g,
                                            const Coef &c, int z, int y, int x) {
  const int64_t p = gidx(g, z, y, x);
  const float uc = u[p];
  auto nb = [&](int ax, int k) {
    return u[p + (ax == 2 ? (int64_t)k : ax == 1 ? (int64_t)k * g.px : (int64_t)k * g.plane)];
  };
  const float lap = plain_lap<R, THREE_D, decltype(nb), ISO2>(uc, c, nb);
  if (EQ == kAcoustic) {
    un[p] = leapfrog(A[p], C[p], uc, un[p], lap);
  } else {
    const bool interior = !g.hold || (x > 0 && x < g.n2 - 1 && y > 0 && y < g.n1 - 1 &&
                                      (!THREE_D || (z > 0 && z < g.n0 - 1)));
    if (interior) un[p] = uc + lap;
  }
}

template <int R, int EQ, bool THREE_D, bool ISO2 = false>
__global__ void __launch_bounds__(256)
k_stencil_plain(const float *__restrict__ u, float *un, const float *__restrict__ A,
                const float *__restrict__ C, Geom g, Coef c) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.n2 || y >= g.n1) return;
  plain_point<R, EQ, THREE_D, ISO2>(u, un, A, C, g, c, z, y, x);
}

// ---------------------------------------------------------------------------
// 2-D step streamed along y.  A warp owns a strip of 64·NP columns (a lane per pair
// of adjacent x points, or with NP = 2 per four adjacent points, read from shared
// memory 16 bytes at a time) and a segment of rows [ya, yb).  Rows ya-R .. yb+R-1
// of u^n (with the x halo) are copied into the warp's ring in shared memory with
// cp.async, s2_d(R) rows ahead of the row in use, so many bytes stay in flight (one
// thread per point keeps too few to fill HBM on large grids).  Each arriving row's
// values at the lane's pairs enter a register queue of 2R+1 rows; R rows later the
// warp updates the middle row: the y part of the Laplacian from the queue, the x
// part from that row's staged copy, still in the ring.  The per-point operation
// sequence is plain_lap's and plain_point's (packed FP32x2 over the pair: each
// lane the scalar round-to-nearest operation), so results are bitwise the plain
// kernel's.  Warps are independent streams; neighbouring strips of a segment run
// together, so the halo columns they share come from L2.
// ---------------------------------------------------------------------------
constexpr int kS2W = 64;  // strip width (columns) a pair a lane
__host__ __device__ constexpr int s2_hx(int R) { return (R + 3) / 4 * 4; }  // x halo, 16-B multiple
__host__ __device__ constexpr int s2_rw(int R, int P = 1) {  // staged row (floats), P pairs a lane
  return kS2W * P + 2 * s2_hx(R);
}
// ring rows per warp: a multiple of the queue length 2R+1 (an unrolled group of that
// many rows then addresses ring and queue slots statically) holding the R rows back
// to the one being updated, the row in use and about 8 rows in flight.  Above radius
// 4 one queue length: the loop is unrolled over the ring, and two queue lengths of a
// radius-8 body overflowed the instruction cache ("no instruction" the top stall);
// there the step is compute-bound and 4-7 rows in flight are enough
__host__ __device__ constexpr int s2_nr(int R) {
  return R > 4 ? 2 * R + 1 : (2 * R + 1) * ((R + 2 + 8 + 2 * R) / (2 * R + 1));
}
__host__ __device__ constexpr int s2_d(int R) {  // rows in flight
  return s2_nr(R) - R - 2 < 10 ? s2_nr(R) - R - 2 : 10;
}
// warps (streams) per block: 8, or 4 above radius 4 (registers and the ring)
__host__ __device__ constexpr int s2_warps(int R) { return R <= 4 ? 8 : 4; }
__host__ __device__ constexpr int s2_smem(int R, int P = 1) {
  return s2_warps(R) * s2_nr(R) * s2_rw(R, P) * 4;
}
// blocks an SM the registers are sized for: four points a lane up to radius 4 keep
// two blocks of 8 warps (128 registers a thread)
__host__ __device__ constexpr int s2_minb(int R, int P) { return P == 2 && R <= 4 ? 2 : 1; }

__device__ __forceinline__ uint32_t s2_saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// 16 bytes global -> shared, asynchronous; src_bytes = 0 fills zeros without reading
__device__ __forceinline__ void s2_copy16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s2_saddr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void s2_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void s2_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int R, int EQ, bool ISO2 = false, int NP = 1>
__global__ void __launch_bounds__(s2_warps(R) * 32, s2_minb(R, NP))
k_stencil2d_stream(const float *__restrict__ u, float *un, const float *__restrict__ A,
                   const float *__restrict__ C, Geom g, Coef c, int nseg, int seglen) {
  constexpr int HX = s2_hx(R), RW = s2_rw(R, NP), NR = s2_nr(R), Q = 2 * R + 1, D = s2_d(R);
  constexpr int W = kS2W * NP;  // strip width
  constexpr int NWP = s2_warps(R);
  constexpr int PH = (R + 1) / 2;  // x pairs each side of the lane's own
  constexpr bool AC = EQ == kAcoustic;
  static_assert(NR % Q == 0 && NR >= D + R + 2, "ring holds the rows in flight and in use");
  static_assert(NP == 1 || NP == 2, "one pair or four adjacent points a lane");
  extern __shared__ __align__(16) float s2_ring[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int strips = (g.n2 + W - 1) / W;
  const int item = blockIdx.x * NWP + warp;
  if (item >= strips * nseg) return;
  const int strip = item % strips, seg = item / strips;  // neighbouring strips together
  const int x0 = strip * W;
  const int ya = seg * seglen, yb = min(g.n1, ya + seglen);
  if (ya >= yb) return;
  float *rg = s2_ring + (size_t)warp * NR * RW;
  const int T = (yb - ya) + 2 * R;  // rows streamed: ya-R .. yb+R-1
  // padded offset of (row ya - R, column x0 - HX); rows -R .. n1+R-1 exist
  const float *src0 = u + gidx(g, 0, ya - R, x0) - HX;
  const int col0 = x0 + kHaloX - HX;  // padded column of the staged row's first float
  auto issue = [&](int t) {           // row ya - R + t into ring slot t % NR
    if (t < T) {
      float *dst = rg + (t % NR) * RW;
      const float *src = src0 + (int64_t)t * g.px;
#pragma unroll
      for (int ch = lane; ch < RW / 4; ch += 32) {
        const bool in = col0 + 4 * ch + 4 <= g.px;  // past the row pitch: zeros, never used
        s2_copy16(dst + 4 * ch, in ? src + 4 * ch : src, in ? 16 : 0);
      }
    }
    s2_commit();  // an empty group past the end keeps the wait count fixed
  };
  const bool hold = !AC && g.hold;
  constexpr int LW = 2 * NP;  // points a lane: its pairs p at x0 + LW·lane + 2p
  constexpr int CH = HX / 4;  // 16-byte chunks of the staged row each side of a lane's four
  bool xin0[NP], xin1[NP];    // the points of pair p to update
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int x = x0 + LW * lane + 2 * p;
    xin0[p] = hold ? (x > 0 && x < g.n2 - 1) : x < g.n2;
    xin1[p] = hold ? (x + 1 > 0 && x + 1 < g.n2 - 1) : x + 1 < g.n2;
  }
  float2 q[NP][Q];  // u^n at pair p, row t in slot t % Q
#pragma unroll
  for (int t = 0; t < D; ++t) issue(t);
  for (int tb = 0; tb < T; tb += NR) {
#pragma unroll
    for (int ph = 0; ph < NR; ++ph) {
      const int t = tb + ph;
      if (t >= T) break;
      issue(t + D);
      s2_wait<D>();  // row t's copies (all but the newest D groups) have landed
      __syncwarp();
      if constexpr (NP == 1) {
        q[0][ph % Q] = *reinterpret_cast<const float2 *>(rg + ph * RW + HX + 2 * lane);
      } else {
        const float4 v = *reinterpret_cast<const float4 *>(rg + ph * RW + HX + 4 * lane);
        q[0][ph % Q] = make_float2(v.x, v.y);
        q[1][ph % Q] = make_float2(v.z, v.w);
      }
      if (t >= 2 * R) {  // row y = ya + t - 2R: its y neighbours are all in the queue
        const int y = ya + t - 2 * R;
        const bool yin = hold ? (y > 0 && y < g.n1 - 1) : true;
        const float *rr = rg + ((ph + NR - R) % NR) * RW + HX + LW * lane;  // row y, staged
        float2 xp[NP == 1 ? 2 * PH + 1 : 1];  // one pair: the row's pairs around its own
        float4 xc[NP == 1 ? 1 : 2 * CH + 1];  // four points: the 16-byte chunks around them
        if constexpr (NP == 1) {
#pragma unroll
          for (int d = -PH; d <= PH; ++d) xp[d + PH] = *reinterpret_cast<const float2 *>(rr + 2 * d);
        } else {
#pragma unroll
          for (int d = -CH; d <= CH; ++d) xc[d + CH] = *reinterpret_cast<const float4 *>(rr + 4 * d);
        }
        auto xv = [&](int i) -> float {  // four points: u at the lane's first x + i
          const int j = i + 4 * CH;
          const float4 &c4 = xc[j >> 2];
          return (j & 3) == 0 ? c4.x : (j & 3) == 1 ? c4.y : (j & 3) == 2 ? c4.z : c4.w;
        };
        float2 val[NP];  // u^{n+1} at the lane's pairs
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const int x = x0 + LW * lane + 2 * p;
          const float2 ucy = q[p][(ph + Q - R) % Q];
          float2 lap = make_float2(0.f, 0.f);
          // u(x+k) + u(x-k) at the pair: aligned pairs for even k, halves of the
          // neighbouring pairs for odd k
          auto xsum = [&](int k) -> float2 {
            if constexpr (NP == 1) {
              if ((k & 1) == 0) return __fadd2_rn(xp[PH + k / 2], xp[PH - k / 2]);
              return make_float2(__fadd_rn(xp[PH + (k - 1) / 2].y, xp[PH - (k + 1) / 2].y),
                                 __fadd_rn(xp[PH + (k + 1) / 2].x, xp[PH - (k - 1) / 2].x));
            } else {
              const int o = 2 * p;
              if ((k & 1) == 0)
                return __fadd2_rn(make_float2(xv(o + k), xv(o + k + 1)),
                                  make_float2(xv(o - k), xv(o - k + 1)));
              return make_float2(__fadd_rn(xv(o + k), xv(o - k)),
                                 __fadd_rn(xv(o + 1 + k), xv(o + 1 - k)));
            }
          };
          auto ysum = [&](int k) -> float2 {  // u(y+k) + u(y-k) from the queue
            return __fadd2_rn(q[p][(ph + Q - R + k) % Q], q[p][(ph + 2 * Q - R - k) % Q]);
          };
          if constexpr (ISO2) {  // plain_lap's equal-spacing form
            const float2 nuc4 = make_float2(-4.f * ucy.x, -4.f * ucy.y);
#pragma unroll
            for (int k = 1; k <= R; ++k)
              lap = __ffma2_rn(c.wp[2][k], __fadd2_rn(__fadd2_rn(ysum(k), xsum(k)), nuc4), lap);
          } else {
            const float2 nuc2 = make_float2(-(ucy.x + ucy.x), -(ucy.y + ucy.y));
#pragma unroll
            for (int k = 1; k <= R; ++k) lap = __ffma2_rn(c.wp[1][k], __fadd2_rn(ysum(k), nuc2), lap);
#pragma unroll
            for (int k = 1; k <= R; ++k) lap = __ffma2_rn(c.wp[2][k], __fadd2_rn(xsum(k), nuc2), lap);
          }
          const int64_t pi = gidx(g, 0, y, x);
          if (AC) {
            float2 prev, a, cc;
            if (xin0[p] && xin1[p]) {
              prev = *reinterpret_cast<const float2 *>(un + pi);
              a = *reinterpret_cast<const float2 *>(A + pi);
              cc = *reinterpret_cast<const float2 *>(C + pi);
            } else {
              prev = make_float2(xin0[p] ? un[pi] : 0.f, xin1[p] ? un[pi + 1] : 0.f);
              a = make_float2(xin0[p] ? A[pi] : 0.f, xin1[p] ? A[pi + 1] : 0.f);
              cc = make_float2(xin0[p] ? C[pi] : 0.f, xin1[p] ? C[pi + 1] : 0.f);
            }
            val[p] = make_float2(leapfrog(a.x, cc.x, ucy.x, prev.x, lap.x),
                                 leapfrog(a.y, cc.y, ucy.y, prev.y, lap.y));
          } else {
            val[p] = make_float2(ucy.x + lap.x, ucy.y + lap.y);
          }
        }
        // the four points in one 16-byte store where all are updated (x a multiple of 4,
        // row pitch and x halo multiples of 32 floats: aligned), else point by point
        if (yin) {
          const int64_t pi = gidx(g, 0, y, x0 + LW * lane);
          if (NP == 2 && xin0[0] && xin1[0] && xin0[NP - 1] && xin1[NP - 1]) {
            *reinterpret_cast<float4 *>(un + pi) =
                make_float4(val[0].x, val[0].y, val[NP - 1].x, val[NP - 1].y);
          } else {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              if (xin0[p] && xin1[p])
                *reinterpret_cast<float2 *>(un + pi + 2 * p) = val[p];
              else {
                if (xin0[p]) un[pi + 2 * p] = val[p].x;
                if (xin1[p]) un[pi + 2 * p + 1] = val[p].y;
              }
            }
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Two diffusion steps in one pass of the row stream (radius 1 and 2, zero halo):
// u^{n+2} from u^n, reading u^n once and writing u^{n+2} once, 4 instead of 8
// bytes a point-step.  A warp streams the rows ya-2R .. yb+2R-1 of u^n into its
// ring A as k_stencil2d_stream does; for each arriving row t it computes the
// intermediate row i = t-R of u^{n+1} on 64 columns, its 60-column strip widened by
// 2 each side (every lane a pair, lanes 0 and 31 the widening: no divergent edge
// work), into ring B (2R+1 rows, shared memory) and
// into a register queue of the lane's pair, and from those the row o = i-R of
// u^{n+2}.  Both stages run plain_lap's operation sequence and plain_point's
// update, and the intermediate values follow the single step's rules (zero
// outside the grid, boundary nodes held when g.hold), so the result is bitwise
// two launches of the one-step kernels.  Rows of u^n further than R outside the
// grid (needed only by intermediate rows outside it, which are zero) are not
// read.  The caller writes into the other level: u^{n+1} is never stored.
// ---------------------------------------------------------------------------
// P pairs a lane (halves of 64 columns of the widened strip): a warp outputs 64P-4
// columns (a multiple of 4) from staged rows 64P + 2·HX wide
__host__ __device__ constexpr int s2t_w(int P) { return 64 * P - 4; }
__host__ __device__ constexpr int s2t_rw(int R, int P) { return 64 * P + 2 * s2_hx(R); }
__host__ __device__ constexpr int s2t_nr(int R) {  // ring A rows: a multiple of 2R+1
  return (2 * R + 1) * ((2 * R + 2 + 8 + 2 * R) / (2 * R + 1));
}
__host__ __device__ constexpr int s2t_d(int R) { return s2t_nr(R) - 2 * R - 2; }  // in flight
__host__ __device__ constexpr int s2t_smem(int R, int P) {
  return s2_warps(R) * (s2t_nr(R) + 2 * R + 1) * s2t_rw(R, P) * 4;
}

template <int R, bool ISO2 = false, int NP = 1>
__global__ void __launch_bounds__(s2_warps(R) * 32)
k_stencil2d_stream2(const float *__restrict__ u, float *un, Geom g, Coef c, int nseg, int seglen) {
  constexpr int HX = s2_hx(R), RW = s2t_rw(R, NP), Q = 2 * R + 1, NR = s2t_nr(R), D = s2t_d(R);
  constexpr int kS2P = NP;            // pairs a lane
  constexpr int kS2W2 = s2t_w(kS2P);  // output columns a warp
  constexpr int NWP = s2_warps(R);
  constexpr int PH = (R + 1) / 2;  // x pairs each side of the lane's own
  static_assert(R <= 2 && NR % Q == 0 && D >= 1 && HX == 4 && (kS2P == 1 || kS2P == 2),
                "radius 1-2; the 64·P intermediate columns x0-2 .. x0+64P-3 and their x "
                "neighbours x0-4 .. x0+64P-1 lie in the staged row x0-4 .. x0+64P+3");
  extern __shared__ __align__(16) float s2_ring[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int strips = (g.n2 + kS2W2 - 1) / kS2W2;
  const int item = blockIdx.x * NWP + warp;
  if (item >= strips * nseg) return;
  const int strip = item % strips, seg = item / strips;
  const int x0 = strip * kS2W2;  // the staged rows start at x0 - HX as in k_stencil2d_stream
  const int ya = seg * seglen, yb = min(g.n1, ya + seglen);
  if (ya >= yb) return;
  float *ra = s2_ring + (size_t)warp * (NR + Q) * RW;  // u^n rows
  float *rb = ra + NR * RW;                            // u^{n+1} rows, slot i mod Q
  const int T = (yb - ya) + 4 * R;  // rows streamed: ya-2R .. yb+2R-1
  const int col0 = x0 + kHaloX - HX;
  auto issue = [&](int t) {  // row ya - 2R + t into ring slot t % NR
    if (t < T) {
      const int r = ya - 2 * R + t;
      const bool row_in = r >= -R && r < g.n1 + R;  // rows of the padded layout
      float *dst = ra + (t % NR) * RW;
      const float *src = row_in ? u + gidx(g, 0, r, x0) - HX : u;
#pragma unroll
      for (int ch = lane; ch < RW / 4; ch += 32) {
        const bool in = row_in && col0 + 4 * ch + 4 <= g.px;
        s2_copy16(dst + 4 * ch, in ? src + 4 * ch : u, in ? 16 : 0);
      }
    }
    s2_commit();
  };
  const bool hold = g.hold != 0;
  // one step at a pair from its centre value, a y-sum accessor and the row's pairs
  // around it: plain_lap's sequence (ISO2: one weight per offset), then uc + lap
  auto lap_pair = [&](float2 uc, auto ysum, const float2 *xp) -> float2 {
    auto xsum = [&](int k) -> float2 {
      if ((k & 1) == 0) return __fadd2_rn(xp[PH + k / 2], xp[PH - k / 2]);
      return make_float2(__fadd_rn(xp[PH + (k - 1) / 2].y, xp[PH - (k + 1) / 2].y),
                         __fadd_rn(xp[PH + (k + 1) / 2].x, xp[PH - (k - 1) / 2].x));
    };
    float2 lap = make_float2(0.f, 0.f);
    if constexpr (ISO2) {
      const float2 nuc4 = make_float2(-4.f * uc.x, -4.f * uc.y);
#pragma unroll
      for (int k = 1; k <= R; ++k)
        lap = __ffma2_rn(c.wp[2][k], __fadd2_rn(__fadd2_rn(ysum(k), xsum(k)), nuc4), lap);
    } else {
      const float2 nuc2 = make_float2(-(uc.x + uc.x), -(uc.y + uc.y));
#pragma unroll
      for (int k = 1; k <= R; ++k) lap = __ffma2_rn(c.wp[1][k], __fadd2_rn(ysum(k), nuc2), lap);
#pragma unroll
      for (int k = 1; k <= R; ++k) lap = __ffma2_rn(c.wp[2][k], __fadd2_rn(xsum(k), nuc2), lap);
    }
    return make_float2(uc.x + lap.x, uc.y + lap.y);
  };
  // the lane's pairs, one in each 64-column half of the widened strip: pair p at x[p] =
  // x0 - 2 + 64p + 2·lane; every pair but the strip's first and last owns output columns
  int x[kS2P], xo[kS2P];
  bool xin0[kS2P], xin1[kS2P], cin0[kS2P], cin1[kS2P], cbd0[kS2P], cbd1[kS2P], cfree[kS2P];
#pragma unroll
  for (int p = 0; p < kS2P; ++p) {
    x[p] = x0 - 2 + 64 * p + 2 * lane;
    xo[p] = 64 * p + 2 * lane - 2;  // the pair's offset from x0 in the staged rows
    const bool own = !(p == 0 && lane == 0) && !(p == kS2P - 1 && lane == 31);
    xin0[p] = own && (hold ? (x[p] > 0 && x[p] < g.n2 - 1) : x[p] < g.n2);
    xin1[p] = own && (hold ? (x[p] + 1 > 0 && x[p] + 1 < g.n2 - 1) : x[p] + 1 < g.n2);
    // the intermediate level's column rules (zero outside the grid, held boundary)
    cin0[p] = x[p] >= 0 && x[p] < g.n2;
    cin1[p] = x[p] + 1 >= 0 && x[p] + 1 < g.n2;
    cbd0[p] = hold && (x[p] == 0 || x[p] == g.n2 - 1);
    cbd1[p] = hold && (x[p] + 1 == 0 || x[p] + 1 == g.n2 - 1);
    cfree[p] = cin0[p] && cin1[p] && !cbd0[p] && !cbd1[p];  // updated on inner rows
  }
  const int ylo = hold ? 1 : 0;  // inner rows ylo .. ylo+yspan-1
  const unsigned yspan = (unsigned)(hold ? g.n1 - 2 : g.n1);
  // the intermediate level at row y of pair p (the single step's rules)
  auto settle = [&](int p, int y, float2 uc, float2 v) -> float2 {
    if (cfree[p] && (unsigned)(y - ylo) < yspan) return v;
    float2 out = make_float2(0.f, 0.f);
    if (y >= 0 && y < g.n1) {
      const bool ybd = hold && (y == 0 || y == g.n1 - 1);
      if (cin0[p]) out.x = (ybd || cbd0[p]) ? uc.x : v.x;
      if (cin1[p]) out.y = (ybd || cbd1[p]) ? uc.y : v.y;
    }
    return out;
  };
  float2 qa[kS2P][Q];  // u^n at pair p, row t in slot t % Q
  float2 qb[kS2P][Q];  // u^{n+1} at pair p, intermediate row of stream position t in slot t % Q
  // ring B's columns outside those stage 1 writes are read (and discarded) by the edge
  // pairs' stage 2: zero them once so that every shared-memory read is of written data
  for (int k = lane; k < Q * RW; k += 32) rb[k] = 0.f;
  __syncwarp();
#pragma unroll
  for (int t = 0; t < D; ++t) issue(t);
  for (int tb = 0; tb < T; tb += NR) {
#pragma unroll
    for (int ph = 0; ph < NR; ++ph) {
      const int t = tb + ph;
      if (t >= T) break;
      issue(t + D);
      s2_wait<D>();  // row t's copies have landed
      __syncwarp();
#pragma unroll
      for (int p = 0; p < kS2P; ++p)
        qa[p][ph % Q] = *reinterpret_cast<const float2 *>(ra + ph * RW + HX + xo[p]);
      if (t >= 2 * R) {
        // stage 1: row i = t-R of u^{n+1} (stream row ya-3R+t) on the widened strip
        const int i = ya - 3 * R + t;
        const float *ri = ra + ((ph + NR - R) % NR) * RW + HX;  // row i of u^n, staged
        float *wb = rb + (ph % Q) * RW + HX;
#pragma unroll
        for (int p = 0; p < kS2P; ++p) {
          float2 xp[2 * PH + 1];
#pragma unroll
          for (int d = -PH; d <= PH; ++d)
            xp[d + PH] = *reinterpret_cast<const float2 *>(ri + xo[p] + 2 * d);
          const float2 uc = qa[p][(ph + Q - R) % Q];
          auto ysum = [&](int k) -> float2 {
            return __fadd2_rn(qa[p][(ph + Q - R + k) % Q], qa[p][(ph + 2 * Q - R - k) % Q]);
          };
          const float2 v = settle(p, i, uc, lap_pair(uc, ysum, xp));
          qb[p][ph % Q] = v;
          *reinterpret_cast<float2 *>(wb + xo[p]) = v;
        }
      }
      __syncwarp();  // ring B row i visible to the warp
      if (t >= 4 * R) {
        // stage 2: row o = i-R of u^{n+2} (stream row ya-4R+t) on the strip; the edge
        // pairs compute with ring B's zeroed edge columns and store nothing
        const int o = ya - 4 * R + t;
        const float *ro = rb + ((ph + Q - R) % Q) * RW + HX;  // row o of u^{n+1}
        const bool yin = hold ? (o > 0 && o < g.n1 - 1) : true;
#pragma unroll
        for (int p = 0; p < kS2P; ++p) {
          float2 xp[2 * PH + 1];
#pragma unroll
          for (int d = -PH; d <= PH; ++d)
            xp[d + PH] = *reinterpret_cast<const float2 *>(ro + xo[p] + 2 * d);
          const float2 vc = qb[p][(ph + Q - R) % Q];
          auto ysum = [&](int k) -> float2 {
            return __fadd2_rn(qb[p][(ph + Q - R + k) % Q], qb[p][(ph + 2 * Q - R - k) % Q]);
          };
          const float2 val = lap_pair(vc, ysum, xp);
          if (yin) {
            const int64_t q = gidx(g, 0, o, x[p]);
            if (xin0[p] && xin1[p])
              *reinterpret_cast<float2 *>(un + q) = val;
            else {
              if (xin0[p]) un[q] = val.x;
              if (xin1[p]) un[q + 1] = val.y;
            }
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Layout moves between dense interior arrays and the padded layout.
// ---------------------------------------------------------------------------
__global__ void k_scatter(const float *__restrict__ dense, float *__restrict__ padded, Geom g) {
  const int64_t n = (int64_t)g.n0 * g.n1 * g.n2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.n2);
    const int64_t r = i / g.n2;
    const int y = (int)(r % g.n1);
    const int z = (int)(r / g.n1);
    padded[gidx(g, z, y, x)] = dense[i];
  }
}

__global__ void k_gather(const float *__restrict__ padded, float *__restrict__ dense, Geom g) {
  const int64_t n = (int64_t)g.n0 * g.n1 * g.n2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.n2);
    const int64_t r = i / g.n2;
    const int y = (int)(r % g.n1);
    const int z = (int)(r / g.n1);
    dense[i] = padded[gidx(g, z, y, x)];
  }
}

// ---------------------------------------------------------------------------
// Acoustic coefficients, once per model, in FP32 with correctly rounded
// divisions (about one ulp from the exact values; C is exactly 1 where damp = 0):
//   σ = damp·dt/2,  A = dt²/(m+σ),  C = (m−σ)/(m+σ).
// stats[0]: min over m of its bit pattern (m > 0 → ordered like the value),
// stats[1]: set when some m ≤ 0 or non-finite, or some damp < 0 or non-finite.
// ---------------------------------------------------------------------------
__global__ void k_coefficients(const float *__restrict__ m, const float *__restrict__ damp,
                               float *__restrict__ A, float *__restrict__ C, Geom g, double dt,
                               unsigned *stats) {
  const int64_t n = (int64_t)g.n0 * g.n1 * g.n2;
  const float dt2 = (float)(dt * dt), half_dt = (float)(0.5 * dt);
  unsigned local_min = 0x7f800000u, bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float mf = m[i];
    const float df = damp ? damp[i] : 0.f;
    if (!(mf > 0.f) || !isfinite(mf) || !(df >= 0.f) || !isfinite(df)) bad = 1;
    local_min = min(local_min, __float_as_uint(mf));
    const float sig = df * half_dt;
    const int x = (int)(i % g.n2);
    const int64_t r = i / g.n2;
    const int y = (int)(r % g.n1);
    const int z = (int)(r / g.n1);
    const int64_t p = gidx(g, z, y, x);
    A[p] = __fdiv_rn(dt2, mf + sig);
    C[p] = __fdiv_rn(mf - sig, mf + sig);
  }
  // warp-reduce before the atomics
  for (int o = 16; o > 0; o >>= 1) {
    local_min = min(local_min, __shfl_xor_sync(0xffffffffu, local_min, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&stats[0], local_min);
    if (bad) atomicOr(&stats[1], 1u);
  }
}

// Source scales w·dt²/m(node) in double, rounded once.
__global__ void k_source_scales(const int64_t *__restrict__ dense_node, const double *__restrict__ w,
                                const float *__restrict__ m, float *__restrict__ scale, int n,
                                double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) scale[i] = (float)(w[i] * dt * dt / (double)m[dense_node[i]]);
}

// ---------------------------------------------------------------------------
// Step counter: kernels of step j in a chunk read n = *step + j.
// ---------------------------------------------------------------------------
__global__ void k_set_step(int64_t *step, int64_t n) { *step = n; }
__global__ void k_advance_step(int64_t *step, int by) { *step += by; }

// ---------------------------------------------------------------------------
// Sparse operators.  NC = 2^D corners per point.
// Injection: un[node] += scale · s_j(t_n) (atomics: sources may share nodes).
// Interpolation: rec[n+1][k] = Σ_c w_kc · un[node_kc]; NC lanes per receiver,
// reduced with warp shuffles.  Every lane of a warp must take part.
// ---------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ void interp_group_store(const float *un, const int64_t *__restrict__ roff,
                                                   const float *__restrict__ rw, float *rec,
                                                   int64_t row, int nrec, int k, int c) {
  float v = 0.f;
  if (k < nrec) v = rw[k * NC + c] * un[roff[k * NC + c]];
  // lanes are corners, axis 0 the highest bit: pairs along the last axis first,
  // the two halves along axis 0 last, so a sum split between two z-slabs (each
  // adding only its own corners, zero for the others) is exactly this sum
#pragma unroll
  for (int o = 1; o < NC; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (c == 0 && k < nrec) rec[row * nrec + k] = v;
}

template <int NC>
__global__ void k_inject(float *un, const int64_t *__restrict__ step, int j, int nsrc,
                         const int64_t *__restrict__ soff, const float *__restrict__ sscale,
                         const float *__restrict__ wav) {
  const int64_t n = *step + j;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsrc * NC) atomicAdd(un + soff[i], sscale[i] * wav[n * nsrc + i / NC]);
}

// FWI misfit of one shot over `rows` trace rows of nrec receivers: r = rec − d_obs
// (float, as recorded), adj_wav row j = r row rows−1−j for j = 0..rows−2 (the adjoint
// source: the residual time reversed; may be null), and part[block] = Σ r² in double
// over the elements the block visits, in a fixed order (blockDim must be 256).
__global__ void k_residual(const float *__restrict__ rec, const float *__restrict__ d_obs,
                           float *__restrict__ adj_wav, int64_t rows, int nrec,
                           double *__restrict__ part) {
  __shared__ double sh[256];
  const int64_t n = rows * nrec;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float r = __fsub_rn(rec[i], d_obs[i]);
    acc = fma((double)r, (double)r, acc);
    const int64_t row = i / nrec;
    if (adj_wav && row >= 1) adj_wav[(rows - 1 - row) * nrec + (i - row * nrec)] = r;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// *out = ½ Σ part[0..n) in a fixed order (one block of 256 threads): J = ½ ||r||².
__global__ void k_sum_partials(const double *__restrict__ part, int n, double *out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * sh[0];
}

// acc[i] += part[i] (the partial traces of one z-slab added into the whole grid's).
__global__ void k_accumulate(float *__restrict__ acc, const float *__restrict__ part, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc[i] += part[i];
}

// rec row = *step + j + 1 (j = -1 with *step = 0 records row 0).
template <int NC>
__global__ void k_interp(const float *un, const int64_t *__restrict__ step, int j, int nrec,
                         const int64_t *__restrict__ roff, const float *__restrict__ rw,
                         float *rec) {
  const int64_t n = *step + j;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  interp_group_store<NC>(un, roff, rw, rec, n + 1, nrec, t / NC, t % NC);
}

}  // namespace fdk

namespace fdk {

// ---------------------------------------------------------------------------
// Batched shots.  At batch tick t a member is at global step step0 + t with
// u^n in level[cur0 ^ (t & 1)]; it writes u^{n+1} into the other level.
// ---------------------------------------------------------------------------
struct MemberDesc {
  float *level[2];
  const float *A, *C;
  Geom g;
  Coef c;
  int cur0;
  int64_t step0;
  int64_t blk0;      // first block of this member in the batched 2-D grid
  int blocks_x;      // blocks along x (2-D members)
  const int64_t *src_off;
  const float *src_scale, *wav;
  int nsrc, nc;
  const int64_t *rec_off;
  const float *rec_w;
  float *rec;
  int nrec;
};

// One step of every 2-D member: blocks of 32 × 8 points, block -> member by
// binary search over blk0 (the plain per-point update: on these L2-resident grids
// it is faster than the staged tile kernel).  The batch kernels run tick *tick + j
// (j: the tick's
// place in a captured chunk).
template <int R>
__global__ void __launch_bounds__(256)
k_stencil2d_batch(const MemberDesc *__restrict__ d, int n, const int64_t *tick, int j) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (d[mid].blk0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const MemberDesc &m = d[lo];
  const int64_t b = blockIdx.x - m.blk0;
  const int x = (int)(b % m.blocks_x) * 32 + threadIdx.x;
  const int y = (int)(b / m.blocks_x) * 8 + threadIdx.y;
  if (x >= m.g.n2 || y >= m.g.n1) return;
  const int par = m.cur0 ^ (int)((*tick + j) & 1);
  if (m.c.iso2)  // per member (a block holds one member's points)
    plain_point<R, kAcoustic, false, true>(m.level[par], m.level[par ^ 1], m.A, m.C, m.g, m.c, 0,
                                           y, x);
  else
    plain_point<R, kAcoustic, false>(m.level[par], m.level[par ^ 1], m.A, m.C, m.g, m.c, 0, y, x);
}

// Source corners of the 2-D members: entry = (member, corner).
__global__ void k_inject_batch(const int2 *__restrict__ e, int n, const MemberDesc *__restrict__ d,
                               const int64_t *tick, int j) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const MemberDesc &m = d[e[i].x];
  const int k = e[i].y;
  const int64_t t = *tick + j;
  float *un = m.level[m.cur0 ^ (int)(t & 1) ^ 1];
  atomicAdd(un + m.src_off[k], m.src_scale[k] * m.wav[(m.step0 + t) * m.nsrc + k / m.nc]);
}

// Receivers of every member: entry = (member, receiver); 8 lanes per receiver
// (lanes beyond the member's 2^D corners add zero), shuffle reduction.
__global__ void k_interp_batch(const int2 *__restrict__ e, int n, const MemberDesc *__restrict__ d,
                               const int64_t *tick, int j) {
  const int64_t tk = *tick + j;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = t >> 3, c = t & 7;
  float v = 0.f;
  const MemberDesc *m = nullptr;
  int k = 0;
  if (r < n) {
    m = &d[e[r].x];
    k = e[r].y;
    if (c < m->nc) {
      const float *un = m->level[m->cur0 ^ (int)(tk & 1) ^ 1];
      v = m->rec_w[k * m->nc + c] * un[m->rec_off[k * m->nc + c]];
    }
  }
  // the order of interp_group_store (lanes past a 2-D member's corners add zero last)
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (r < n && c == 0) m->rec[(m->step0 + tk + 1) * m->nrec + k] = v;
}

}  // namespace fdk

namespace fdk {

// Tile-planes of the pipelined kernel on which C = (m-σ)/(m+σ) is exactly 1
// (σ = 0 at every point: no damping there): flags[tile·n0 + z] = 1.  The kernel
// then skips the C tile and uses 1, which is the value it would have read.
// One block per tile-plane (tile tx × ty points).
__global__ void k_unit_c(const float *__restrict__ C, Geom g, int tiles_x, int tx, int ty,
                         unsigned char *__restrict__ flags) {
  const int64_t tp = blockIdx.x;  // tile * n0 + z
  const int z = (int)(tp % g.n0), tile = (int)(tp / g.n0);
  const int x0 = (tile % tiles_x) * tx, y0 = (tile / tiles_x) * ty;
  int ok = 1;
  for (int i = threadIdx.x; i < tx * ty; i += blockDim.x) {
    const int x = x0 + i % tx, y = y0 + i / tx;
    if (x < g.n2 && y < g.n1 && C[gidx(g, z, y, x)] != 1.f) ok = 0;
  }
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) flags[tp] = (unsigned char)ok;
}

// Odd-reflection boundary (diffusion): before a step, every halo cell at
// distance k = 1..R beyond a boundary node along one axis takes the negated
// value at distance k inside it, u(-k) = -u(k), u(n-1+k) = -u(n-1-k).  Only
// the faces are filled (over the interior of the other axes): the star
// stencil never reads an edge or corner of the halo.  One thread per cell,
// grid-stride; threads run x fastest within a face so rows stay coalesced.
__global__ void k_odd_halo(float *__restrict__ u, Geom g) {
  const int R = g.R;
  const int64_t n0 = g.n0, n1 = g.n1, n2 = g.n2;
  const int64_t f0 = g.R0 ? 2LL * R * n1 * n2 : 0;  // axis-0 faces (3-D only)
  const int64_t f1 = 2LL * R * n0 * n2;             // axis-1 faces
  const int64_t f2 = 2LL * R * n0 * n1;             // axis-2 faces
  const int64_t total = f0 + f1 + f2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = t;
    int z, y, x, zs, ys, xs;
    if (s < f0) {  // [side][k][y][x]
      x = (int)(s % n2); s /= n2;
      y = (int)(s % n1); s /= n1;
      const int k = (int)(s % R) + 1, side = (int)(s / R);
      z = side ? (int)n0 - 1 + k : -k;
      zs = side ? (int)n0 - 1 - k : k;
      ys = y;
      xs = x;
    } else if ((s -= f0) < f1) {  // [z][side][k][x]
      x = (int)(s % n2); s /= n2;
      const int k = (int)(s % R) + 1; s /= R;
      const int side = (int)(s % 2);
      z = (int)(s / 2);
      y = side ? (int)n1 - 1 + k : -k;
      ys = side ? (int)n1 - 1 - k : k;
      zs = z;
      xs = x;
    } else {  // [z][y][side][k]
      s -= f1;
      const int k = (int)(s % R) + 1; s /= R;
      const int side = (int)(s % 2); s /= 2;
      y = (int)(s % n1);
      z = (int)(s / n1);
      x = side ? (int)n2 - 1 + k : -k;
      xs = side ? (int)n2 - 1 - k : k;
      zs = z;
      ys = y;
    }
    u[gidx(g, z, y, x)] = -u[gidx(g, zs, ys, xs)];
  }
}

// FWI imaging condition: g[i] += s · ν(i) · (u⁺(i) − 2u(i) + u⁻(i)) over the
// interior points (g dense, the rest padded), the discrete cross-correlation
// of the adjoint field with the second time difference of the forward field.
__global__ void k_imaging(float *__restrict__ g, const float *__restrict__ nu,
                          const float *__restrict__ up1, const float *__restrict__ u0,
                          const float *__restrict__ um1, Geom geo, float scale) {
  const int64_t n = (int64_t)geo.n0 * geo.n1 * geo.n2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % geo.n2);
    const int64_t r = i / geo.n2;
    const int y = (int)(r % geo.n1);
    const int z = (int)(r / geo.n1);
    const int64_t p = gidx(geo, z, y, x);
    const float d2 = (up1[p] - u0[p]) - (u0[p] - um1[p]);
    g[i] = fmaf(scale * nu[p], d2, g[i]);
  }
}

}  // namespace fdk
