// fd_kernels_tma.cuh -- pipelined 3-D stencil kernel: TMA plane ring + register z-queue.
//
// Work: the grid's (x, y) extent is cut into TX × TY tiles; a "tile-plane" is one
// tile at one z, a "segment" the planes of one tile inside one z-block (ZB
// planes).  Work is ordered z-block-major (inside a block tile by tile, x
// fastest, then z) and shared out over G persistent CTAs (G = SMs × resident
// CTAs) in one of two ways:
//   - equal ranges: every CTA gets the same number of tile-planes to within one
//     (a range may start or end inside a segment);
//   - whole segments: every CTA gets whole segments, at most one CTA per segment.
// Either way CTAs that hold neighbouring tiles stream the same z at about the same
// time, so the halo rows one tile shares with the next are still in L2 when the
// other reads them.  A batch launch (MULTI) takes items {shot, tile, za, zb} from
// a ticket counter instead.
//
// Per CTA: warp NW (the last) is the producer; one lane issues
//   - a TMA load of the u^n plane p (tile plus halo: (TX+2·HXB) × (TY+2R)) into
//     ring U (DU slots), for every p in [za-R, zb+R) of a segment [za, zb);
//   - TMA loads of the u^{n-1}, A, C tiles (TX × TY) of plane p-R into ring X
//     (DX slots) when p-R is a plane the CTA updates (acoustic only).
// The NW consumer warps own NY rows each (lane = x; TY = NW·NY), updated in pairs
// with packed FP32x2 arithmetic.  For every plane p they push u^n(p) at their
// points into a register queue of 2R+1 planes, and once the queue holds
// p-2R..p they update plane zc = p-R: z-neighbours from the queue, x- and
// y-neighbours from the shared copy of plane zc (still in ring U), then store
// u^{n+1} with coalesced 128-byte rows.
//
// Every mbarrier wait is bounded (clock64 budget).  On expiry the kernel writes
// an error code and its block index into err[0..1], stops, waits (bounded) for
// its own TMA copies in flight, and returns; fd_read reports FD_ETIMEOUT.
#pragma once

#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cudaTypedefs.h>
#include <functional>
#include <memory>
#include <queue>
#include <vector>

#include "fd_common.cuh"

namespace fdk {

constexpr int kTmaTX = 32;        // tile width in x (one warp of lanes)
constexpr int kTmaNW = 8;         // consumer warps
constexpr int kTmaThreads = (kTmaNW + 1) * 32;
constexpr int kTmaDX = 4;         // slots of the u^{n-1}/A/C ring
constexpr long long kWaitBudget = 1ll << 31;  // clock cycles (~1 s at 2 GHz)

// Tile shape: the consumer warps own NY rows each, so a tile is TX × (NW·NY)
// points.  The register queue holds 2R+1 planes per row, so NY·(2R+1) bounds
// the rows a thread can carry; the default is 4 rows up to radius 4 and 2
// above, and the autotuner may pick the other of {2, 4}.
__host__ __device__ constexpr int tma_ny(int R) { return R <= 4 ? 4 : 2; }   // default rows/thread
__host__ __device__ constexpr int tma_ty(int NY) { return kTmaNW * NY; }      // tile height
__host__ __device__ constexpr int tma_hxb(int R) { return (R + 3) / 4 * 4; }   // x halo, 16-B multiple
__host__ __device__ constexpr int tma_bw(int R) { return kTmaTX + 2 * tma_hxb(R); }  // box width
__host__ __device__ constexpr int tma_bh(int R, int NY) { return tma_ty(NY) + 2 * R; }  // box height
__host__ __device__ constexpr int tma_ubytes(int R, int NY) { return tma_bw(R) * tma_bh(R, NY) * 4; }
__host__ __device__ constexpr int tma_xbytes(int NY) { return kTmaTX * tma_ty(NY) * 4; }
__host__ __device__ constexpr int tma_align128(int b) { return (b + 127) / 128 * 128; }
// Ring U slots: the window needs R + 1 planes (the centre plane for the x/y
// neighbours up to the newest plane entering the queue); the rest is prefetch.
// The acoustic step keeps 3 planes of prefetch (its ring X of (u^{n-1}, A, C)
// tiles holds most bytes in flight); diffusion reads only u^n, so its ring
// grows to about diff_ring(R) bytes (up to 11 planes of prefetch) to keep
// enough bytes in flight per SM for HBM: 100 KB (two CTAs an SM) from radius 3,
// 56 KB below (up to four CTAs an SM, their register count allowing).
__host__ __device__ constexpr int diff_ring(int R) { return (R <= 2 ? 56 : 100) * 1024; }
__host__ __device__ constexpr int du_fill(int R, int slot_bytes) {
  return R + 12 < diff_ring(R) / tma_align128(slot_bytes) ? R + 12
                                                          : diff_ring(R) / tma_align128(slot_bytes);
}
__host__ __device__ constexpr int tma_du(int R, bool acoustic = true, int slot_bytes = 0) {
  return acoustic || du_fill(R, slot_bytes) < R + 4 ? R + 4 : du_fill(R, slot_bytes);
}
// ring X: kTmaDX slots of (u^{n-1}, A, C); with the FWI epilogue 2 slots of
// (u^{n-1}, A, C, d2, g) so two CTAs still fit on an SM
__host__ __device__ constexpr int tma_dx(bool fwi) { return fwi ? 2 : kTmaDX; }
__host__ __device__ constexpr int tma_xn(bool fwi) { return fwi ? 5 : 3; }
// shared memory: barriers (1 KB) | ring U | ring X
__host__ __device__ constexpr int tma_smem_bytes(int R, int NY, bool acoustic, bool fwi = false) {
  return 1024 + tma_du(R, acoustic, tma_ubytes(R, NY)) * tma_align128(tma_ubytes(R, NY)) +
         (acoustic ? tma_dx(fwi) * tma_xn(fwi) * tma_xbytes(NY) : 0);
}
// Consumer loop unrolling: up to radius 4 by the whole window (2R+1 phases,
// queue slots taken mod 2R+1, no register moves); above, by 4 phases with a
// slide of the queue after each group, which keeps the code small enough for
// the instruction cache at the cost of 2R moves per 4 planes and row
__host__ __device__ constexpr int tma_unroll(int R) { return R <= 4 ? 2 * R + 1 : 4; }
// CTAs per SM the register budget is sized for (launch bounds): the queue
// (NY·(2R+1) floats) dominates a consumer thread's registers
__host__ __device__ constexpr int tma_minb(int R, int NY) {
  return NY * (2 * R + 1) <= 20 ? 3 : (NY * (2 * R + 1) <= 40 ? 2 : 1);
}

// ---------------------------------------------------------------------------
// PTX helpers (mbarrier, TMA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false if the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          long long budget = kWaitBudget) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}

// Self-test of the bounded wait: phase 0 of a fresh barrier that nothing
// arrives on never completes, so the wait must give up after `budget` cycles.
__global__ void k_selftest_wait(long long budget, int *out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long t0 = clock64();
  const bool completed = mbar_wait(&bar, 0, budget);
  const long long waited = clock64() - t0;
  if (threadIdx.x == 0) {
    out[0] = completed ? 0 : 1;
    out[1] = (int)(waited >> 10);  // kilo-cycles
  }
}
// TMA load of one box into shared memory, completing on an mbarrier, with an L2
// eviction-priority policy (createpolicy): the halo'd u^n planes are re-read
// by the neighbouring tiles, the u^{n-1}/A/C tiles are not.
__device__ __forceinline__ void tma_load_3d_hint(void *dst, const CUtensorMap *map, int x, int y,
                                                 int z, uint64_t *bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// Contiguous share [q0, q1) of the W tile-planes for CTA b of G.
__device__ __forceinline__ void cta_range(int64_t W, int b, int G, int64_t &q0, int64_t &q1) {
  q0 = W * b / G;
  q1 = W * (b + 1) / G;
}

// Position q (z-block-major order) -> segment: tile, first plane za, end zb
// (the segment ends at the end of the z-block or of the range, whichever is first).
__device__ __forceinline__ void segment_at(int64_t q, int64_t q1, int ntiles, int zblock, int n0,
                                           int &tile, int &za, int &zb) {
  const int64_t per_block = (int64_t)ntiles * zblock;
  const int k = (int)(q / per_block);
  const int64_t r = q - k * per_block;
  const int z0 = k * zblock;
  const int len = min(zblock, n0 - z0);
  tile = (int)(r / len);
  za = z0 + (int)(r % len);
  zb = (int)min((int64_t)(z0 + len), za + (q1 - q));
}

// Point-source injection inside the stencil epilogue.  Entries (source
// corners) are sorted by (tile, plane, source); first[tile * n0 + z] is the
// first entry of that tile at plane z or later.
struct SparseArgs {
  const int4 *entries;     // {x, y, z, corner index}
  const int *first;        // ntiles * n0 + 1 offsets (nullptr: no sources)
  const float *src_scale;  // [nsrc*NC] w·dt²/m(node)
  const float *wav;        // [nt][nsrc]
  const int64_t *step;     // device step counter; this launch is step *step + j
  int j;
  int nsrc, nc;
};

// Where a tensor map's coordinate 0 lies, per axis: the kernels address every
// box by interior coordinates plus these offsets.  Maps over the interior
// (offset 0) let TMA fill the values outside the grid with zeros without reading
// the zero halo from DRAM; a padded axis (offset kHaloX in x, R in y and z) reads
// the halo from memory, where it holds data: the odd-reflection mirror
// (diffusion) or, along z, a neighbouring slab's planes.
struct MapOrigin {
  int ox, oy, oz;
};

struct TmaArgs {
  Geom g;
  Coef c;
  MapOrigin org;     // tensor-map origin of every map of this launch
  int tiles_x;       // tiles along x
  int ntiles;        // tiles in a plane
  int zblock;        // planes per z-block of the work order
  int aligned;       // 1: CTAs take whole (z-block, tile) segments; 0: equal tile-plane ranges
  int64_t W;         // tile-planes
  float *out;        // u^{n+1} (padded layout; the buffer that held u^{n-1})
  int *err;          // err[0] = code, err[1] = block
  SparseArgs sp;
  const unsigned char *unit_c;  // [ntiles * n0]: 1 where C = 1 on the whole tile-plane (or null;
                                // used up to radius 4)
  // FWI epilogue (instances with FWI = true; padded layout, interior points):
  float *d2;           // if set: u^{n+1} - 2u^n + u^{n-1} of this step
  float *img;          // if set: img += img_scale * u^{n+1} * img_d2 (imaging condition)
  const float *img_d2;
  float img_scale;
  // work queue (aligned = 2, x-pair instances with QUEUE = true): {0, tile, za, zb}
  // items, z-layer by z-layer, tile by tile; wq[0] = next ticket, wq[1] = CTAs done
  const int4 *items;
  int nitems;
  unsigned *wq;
};

// The segment at work position q of a CTA's range [q, q1), advancing q.
// Equal tile-plane ranges (aligned = 0): a range may start or end inside a
// segment.  Whole segments (aligned = 1): q counts segments, z-block-major.
__device__ __forceinline__ void next_segment(const TmaArgs &a, int64_t &q, int64_t q1, int &tile,
                                             int &za, int &zb) {
  if (a.aligned) {
    tile = (int)(q % a.ntiles);
    za = (int)(q / a.ntiles) * a.zblock;
    zb = min(a.g.n0, za + a.zblock);
    ++q;
  } else {
    segment_at(q, q1, a.ntiles, a.zblock, a.g.n0, tile, za, zb);
    q += zb - za;
  }
}

// Work queue: the producer lane takes the next item with a ticket; past the last
// item it gets the end mark {-1, ...}.
__device__ __forceinline__ int4 take_item(unsigned *ticket, const int4 *items, int nitems) {
  const unsigned it = atomicAdd(ticket, 1u);
  return it < (unsigned)nitems ? items[it] : make_int4(-1, 0, 0, 0);
}
// Called once per CTA after its producer took its last ticket: the last CTA of the
// launch resets the queue for the next launch (launches of a plan are stream-ordered).
__device__ __forceinline__ void queue_done(unsigned *wq) {
  __threadfence();  // this CTA's tickets before its count
  if (atomicAdd(&wq[1], 1u) == gridDim.x - 1) {
    atomicExch(&wq[0], 0u);
    atomicExch(&wq[1], 0u);
  }
}

// One shot of a batch (device memory, one per member).  At batch tick t the
// shot is at global step step0 + t with u^n in level[cur0 ^ (t & 1)].
struct alignas(64) ShotDesc {
  CUtensorMap map_u[2];   // levels, halo box
  CUtensorMap map_t[2];   // levels, tile box (u^{n-1} reads)
  CUtensorMap map_a, map_c;
  Geom g;
  Coef c;
  MapOrigin org;
  float *level[2];
  int tiles_x, ntiles, zblock, cur0;
  int64_t step0;
  const int4 *entries;     // source corners (see SparseArgs); nullptr: none
  const int *first;
  const float *src_scale;
  const float *wav;
  int nsrc, nc;
};

// Batch work: items {shot, tile, za, zb} ordered z-layer by z-layer (thick
// layers first, thin last), shot by shot, tile by tile; CTAs take them in
// order from a ticket counter, so neighbouring tiles stream in step and the
// last items are short.
struct BatchArgs {
  const ShotDesc *shots;
  const int4 *items;
  int nitems;
  unsigned *ticket;        // [2]: counter of this tick (tick & 1); the other is reset
  const int64_t *tick;     // device tick counter of the batch; this launch runs *tick + j
  int j;
  int *err;
  float2 wp[3][kMaxR + 1];  // weight pairs of every 3-D shot (they share the spacing)
};

// Queue slot of window offset o (0 .. 2R) in phase ph of an unrolled group.
template <int U, int Q>
__device__ __forceinline__ constexpr int tma_qslot(int ph, int o) {
  return U == Q ? (ph + o) % Q : ph + o;
}

// Source corners at tile-plane zc (rare, so kept out of the unrolled loop):
// entries [ecur, eend) are sorted by (tile, plane, source); 32 at a time, one
// per lane, coefficients fetched in parallel; the lane that owns the point
// adds them to its rows (v.x .. v.w) in entry order.  Returns the new cursor
// and the plane of the next entry.
struct SourceHits {
  float4 v;
  int ecur, nxt_z;
};
__device__ __forceinline__ SourceHits source_hits(const int4 *entries, const float *src_scale,
                                                  const float *wav, int nsrc, int nc, int ecur,
                                                  int eend, int zc, int ybase, int ny, int x,
                                                  int lane, int64_t nstep, float4 v) {
  while (true) {
    const int e = ecur + lane;
    const int4 en = e < eend ? entries[e] : make_int4(0, 0, INT_MAX, 0);
    const int cnt = __popc(__ballot_sync(0xffffffffu, en.z == zc));  // a prefix
    const int jr = en.y - ybase;
    const bool here = en.z == zc && jr >= 0 && jr < ny;
    float add = 0.f;
    if (here) add = src_scale[en.w] * wav[nstep * nsrc + en.w / nc];
    unsigned mine = __ballot_sync(0xffffffffu, here);
    while (mine) {
      const int b = __ffs(mine) - 1;
      mine &= mine - 1;
      const int ex = __shfl_sync(0xffffffffu, en.x, b);
      const int ej = __shfl_sync(0xffffffffu, jr, b);
      const float ad = __shfl_sync(0xffffffffu, add, b);
      if (ex == x) {
        if (ej == 0) v.x += ad;
        else if (ej == 1) v.y += ad;
        else if (ej == 2) v.z += ad;
        else v.w += ad;
      }
    }
    ecur += cnt;
    if (cnt < 32) break;
  }
  SourceHits h;
  h.v = v;
  h.ecur = ecur;
  h.nxt_z = ecur < eend ? entries[ecur].z : INT_MAX;
  return h;
}
// Out-of-line copy for the large-radius kernels, whose loop body is the
// biggest; inlined copies there would crowd the instruction cache.
__device__ __noinline__ SourceHits source_hits_call(const int4 *entries, const float *src_scale,
                                                    const float *wav, int nsrc, int nc, int ecur,
                                                    int eend, int zc, int ybase, int ny, int x,
                                                    int lane, int64_t nstep, float4 v) {
  return source_hits(entries, src_scale, wav, nsrc, nc, ecur, eend, zc, ybase, ny, x, lane, nstep,
                     v);
}

// ISO: equal spacing on all axes, so one weight per k multiplies the sum of the
// six neighbours minus 6u (still exact for constants); otherwise one difference
// per axis.  MULTI: the launch steps every shot of a batch (BatchArgs), taking
// work items dynamically; one shot takes static contiguous ranges.
template <int R, int NY, int EQ, bool ISO, bool MULTI, bool FWI = false>
__global__ void __launch_bounds__(kTmaThreads, tma_minb(R, NY))
k_stencil3d_tma(const __grid_constant__ CUtensorMap map_u,   // u^n, halo box
                const __grid_constant__ CUtensorMap map_p,   // u^{n-1}, tile box
                const __grid_constant__ CUtensorMap map_a,   // A, tile box
                const __grid_constant__ CUtensorMap map_c,   // C, tile box
                const __grid_constant__ CUtensorMap map_e,   // FWI: img_d2, tile box
                const __grid_constant__ CUtensorMap map_g,   // FWI: img, tile box
                const TmaArgs args, const BatchArgs bat) {
  constexpr int TY = tma_ty(NY);
  constexpr int HXB = tma_hxb(R), BW = tma_bw(R), DU = tma_du(R, EQ == kAcoustic, tma_ubytes(R, NY));
  constexpr int USLOT = tma_align128(tma_ubytes(R, NY)) / 4;  // floats per ring-U slot
  constexpr int XT = kTmaTX * TY;                          // floats per tile
  constexpr int Q = 2 * R + 1;                             // window of planes
  constexpr int U = tma_unroll(R);                         // phases per unrolled group
  constexpr int QL = U == Q ? Q : Q + U - 1;               // queue registers per row
  constexpr bool kSplit = R > 4;                           // two accumulation chains
  static_assert(NY % 2 == 0, "rows are updated in pairs (packed FP32x2 arithmetic)");
  // skipping the C tile where C = 1 pays on one shot up to radius 4; above, and in
  // the batched kernel, the extra live registers cost more than the bytes saved
  constexpr bool kUnitC = EQ == kAcoustic && !MULTI && R <= 4;
  constexpr int DX = tma_dx(FWI), XN = tma_xn(FWI);        // ring X slots, tiles per slot
  const bool img = FWI && args.img != nullptr;             // imaging inputs in ring X
  constexpr bool AC = EQ == kAcoustic;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *full_u = reinterpret_cast<uint64_t *>(smem);
  uint64_t *empty_u = full_u + DU;
  uint64_t *full_x = empty_u + DU;
  uint64_t *empty_x = full_x + DX;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty_x + DX);
  volatile int4 *item_ring = reinterpret_cast<volatile int4 *>(smem + 512);  // batches: 4 items
  float *ring_u = reinterpret_cast<float *>(smem + 1024);
  float *ring_x = ring_u + DU * USLOT;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int *const err = MULTI ? bat.err : args.err;
  if (threadIdx.x == 0) {
    for (int i = 0; i < DU; ++i) {
      mbar_init(&full_u[i], 1);
      mbar_init(&empty_u[i], kTmaNW);
    }
    for (int i = 0; i < DX; ++i) {
      mbar_init(&full_x[i], 1);
      mbar_init(&empty_x[i], kTmaNW);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  int64_t q0 = 0, q1 = 0;
  if constexpr (!MULTI) {
    if (args.aligned)  // whole segments: q counts (z-block, tile) segments
      cta_range((int64_t)args.ntiles * ((args.g.n0 + args.zblock - 1) / args.zblock), blockIdx.x,
                gridDim.x, q0, q1);
    else
      cta_range(args.W, blockIdx.x, gridDim.x, q0, q1);
  }
  const int64_t tick = MULTI ? *bat.tick + bat.j : 0;
  if constexpr (MULTI) {
    if (blockIdx.x == 0 && threadIdx.x == 0) bat.ticket[(tick + 1) & 1] = 0u;  // next tick's
  }
  int shot = 0;

  if (warp == kTmaNW) {
    // ------------------------------- producer -------------------------------
    if (lane == 0) {
      if constexpr (!MULTI) {
        tma_prefetch_desc(&map_u);
        if (AC) {
          tma_prefetch_desc(&map_p);
          tma_prefetch_desc(&map_a);
          tma_prefetch_desc(&map_c);
        }
      }
      uint32_t su = 0, sx = 0;  // fills issued to rings U and X
      const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
      bool ok = true;
      int64_t q = q0;
      unsigned nitem = 0;        // batches: items taken by this block
      while (ok) {
        int tile, za, zb, tiles_x;
        if constexpr (MULTI) {
          const unsigned it = atomicAdd(&bat.ticket[tick & 1], 1u);
          const int4 item = it < (unsigned)bat.nitems ? bat.items[it] : make_int4(-1, 0, 0, 0);
          item_ring[nitem & 3].x = item.x;
          item_ring[nitem & 3].y = item.y;
          item_ring[nitem & 3].z = item.z;
          item_ring[nitem & 3].w = item.w;
          ++nitem;
          if (item.x < 0) {
            // no work left: complete the next ring-U phase without data so the
            // consumers read the end mark published above
            const uint32_t slot = su % DU;
            if (su >= (uint32_t)DU && !mbar_wait(&empty_u[slot], ((su / DU) - 1) & 1)) {
              ok = false;
              break;
            }
            mbar_arrive(&full_u[slot]);
            ++su;
            break;
          }
          shot = item.x;
          tile = item.y;
          za = item.z;
          zb = item.w;
          tiles_x = bat.shots[shot].tiles_x;
        } else {
          if (q >= q1) break;
          next_segment(args, q, q1, tile, za, zb);
          tiles_x = args.tiles_x;
        }
        const int x0 = (tile % tiles_x) * kTmaTX, y0 = (tile / tiles_x) * TY;
        const CUtensorMap *mu = &map_u, *mp = &map_p, *ma = &map_a, *mc = &map_c;
        const unsigned char *uc_flags = kUnitC ? args.unit_c : nullptr;
        const int n0p = args.g.n0;
        MapOrigin o = args.org;
        if constexpr (MULTI) {
          const ShotDesc &d = bat.shots[shot];
          const int par = d.cur0 ^ (int)(tick & 1);
          mu = &d.map_u[par];
          mp = &d.map_t[par ^ 1];
          ma = &d.map_a;
          mc = &d.map_c;
          o = d.org;
        }
        for (int p = za - R; p < zb + R; ++p) {
          if (*abort_flag) { ok = false; break; }
          const int zc = p - R;
          if (AC && zc >= za) {
            const uint32_t slot = sx % DX;
            if (sx >= (uint32_t)DX && !mbar_wait(&empty_x[slot], ((sx / DX) - 1) & 1)) {
              ok = false;
              break;
            }
            float *dst = ring_x + slot * XN * XT;
            // where C = 1 on the whole tile-plane its tile is not loaded
            const bool cone = kUnitC && uc_flags && uc_flags[(int64_t)tile * n0p + zc];
            mbar_expect_tx(&full_x[slot], ((img ? 5 : 3) - (cone ? 1 : 0)) * XT * 4);
            const int tx = x0 + o.ox, ty = y0 + o.oy, tz = zc + o.oz;  // tile box
            tma_load_3d_hint(dst, mp, tx, ty, tz, &full_x[slot], once);
            tma_load_3d_hint(dst + XT, ma, tx, ty, tz, &full_x[slot], once);
            if (!cone) tma_load_3d_hint(dst + 2 * XT, mc, tx, ty, tz, &full_x[slot], once);
            if (img) {
              tma_load_3d_hint(dst + 3 * XT, &map_e, tx, ty, tz, &full_x[slot], once);
              tma_load_3d_hint(dst + 4 * XT, &map_g, tx, ty, tz, &full_x[slot], once);
            }
            ++sx;
          }
          const uint32_t slot = su % DU;
          if (su >= (uint32_t)DU && !mbar_wait(&empty_u[slot], ((su / DU) - 1) & 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full_u[slot], tma_ubytes(R, NY));
          // halo'd box: x from x0 - HXB, y from y0 - R (interior coordinates)
          tma_load_3d_hint(ring_u + slot * USLOT, mu, x0 - HXB + o.ox, y0 - R + o.oy, p + o.oz,
                           &full_u[slot], keep);
          ++su;
        }
      }
      if (!ok && atomicCAS(err, 0, 2) == 0) err[1] = blockIdx.x;
      if (!ok) *abort_flag = 1;
      // drain: every fill issued must land before the block exits
      bool drained = true;
      for (uint32_t i = 0; i < (uint32_t)DU && i < su; ++i) {
        const uint32_t last = su - 1 - ((su - 1 - i) % DU);  // last fill of slot i
        drained &= mbar_wait(&full_u[last % DU], (last / DU) & 1);
      }
      for (uint32_t i = 0; i < (uint32_t)DX && i < sx; ++i) {
        const uint32_t last = sx - 1 - ((sx - 1 - i) % DX);
        drained &= mbar_wait(&full_x[last % DX], (last / DX) & 1);
      }
      if (!drained && atomicCAS(err, 0, 3) == 0) err[1] = blockIdx.x;
    }
    return;
  }

  // --------------------------------- consumers --------------------------------
  // Fill s of ring U is plane za-R+(s-s0) of the current segment (s0 = its first
  // fill); the warm-up puts planes za-R .. za+R-1 in queue slots 0 .. 2R-1, and
  // the steady loop addresses the window through tma_qslot.
  float2 qp[NY / 2][QL];  // queue, rows paired: .x row 2h, .y row 2h+1
  uint32_t su = 0, sx = 0;
  const int row0 = warp * NY;  // first tile row of this thread
  int64_t nstep = 0;
  if constexpr (!MULTI) nstep = (AC && args.sp.first) ? *args.sp.step + args.sp.j : 0;
  // per-shot parameters (for one shot they stay the kernel's own arguments)
  const float2 *wp0 = args.c.wp[0], *wp1 = args.c.wp[1], *wp2 = args.c.wp[2];
  // weight pair of axis a and offset k, a kernel parameter (the 3-D shots of a
  // batch share their spacing and so their weights)
  auto weight = [&](int a, int k) -> float2 {
    if constexpr (MULTI) return bat.wp[a][k];
    return a == 0 ? wp0[k] : (a == 1 ? wp1[k] : wp2[k]);
  };
  SparseArgs sp = args.sp;
  Geom g = args.g;
  float *out = args.out;
  int64_t q = q0;
  unsigned nitem = 0;
  while (true) {
    int tile, za, zb, tiles_x, n0;
    if constexpr (MULTI) {
      // the next item is published with the first fill of its planes
      if (!mbar_wait(&full_u[su % DU], (su / DU) & 1)) goto timeout;
      const int4 item = make_int4(item_ring[nitem & 3].x, item_ring[nitem & 3].y,
                                  item_ring[nitem & 3].z, item_ring[nitem & 3].w);
      ++nitem;
      if (item.x < 0) break;
      shot = item.x;
      tile = item.y;
      za = item.z;
      zb = item.w;
      tiles_x = bat.shots[shot].tiles_x;
      n0 = bat.shots[shot].g.n0;
    } else {
      if (q >= q1) break;
      next_segment(args, q, q1, tile, za, zb);
      tiles_x = args.tiles_x;
      n0 = args.g.n0;
    }
    if constexpr (MULTI) {
      const ShotDesc &d = bat.shots[shot];
      g = d.g;
      out = d.level[d.cur0 ^ (int)(tick & 1) ^ 1];
      sp.entries = d.entries;
      sp.first = d.first;
      sp.src_scale = d.src_scale;
      sp.wav = d.wav;
      sp.nsrc = d.nsrc;
      sp.nc = d.nc;
      nstep = d.step0 + tick;
    }
    const int x = (tile % tiles_x) * kTmaTX + lane;
    const int ybase = (tile / tiles_x) * TY + row0;
    // tile-planes whose C tile the producer skipped (C = 1 there)
    const unsigned char *ucf = kUnitC ? args.unit_c : nullptr;
    // which of this thread's rows it stores (diffusion: interior nodes only)
    unsigned rows_ok = 0;
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      const int y = ybase + j;
      const bool in = (AC || !g.hold) ? (x < g.n2 && y < g.n1)
                                      : (x > 0 && x < g.n2 - 1 && y > 0 && y < g.n1 - 1);
      rows_ok |= (in ? 1u : 0u) << j;
    }
    float *optr = out + gidx(g, za, ybase, x);
    // sparse entries of this segment: [ecur, eend), next one in a register
    int ecur = 0, eend = 0, nxt_z = INT_MAX;
    if (AC && sp.first) {
      ecur = sp.first[tile * n0 + za];
      eend = sp.first[tile * n0 + zb];
      if (ecur < eend) nxt_z = sp.entries[ecur].z;
    }

    // warm-up: planes za-R .. za+R-1 fill queue slots 0 .. 2R-1
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) {
      const int p = za - R + m;
      const uint32_t slot = su % DU;
      if (!mbar_wait(&full_u[slot], (su / DU) & 1)) goto timeout;
      const float *pl = ring_u + slot * USLOT + (R + row0) * BW + HXB + lane;
#pragma unroll
      for (int h = 0; h < NY / 2; ++h) qp[h][m] = make_float2(pl[2 * h * BW], pl[(2 * h + 1) * BW]);
      if (p < za || p >= zb) {  // plane used for the queue only
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_u[slot]);
      }
      ++su;
    }
    // steady state: update zc = za + i after pushing plane zc + R.  Phase ph
    // of an unrolled group of U: the window of planes zc-R .. zc+R is queue
    // slots ph .. ph+2R (U < Q: slots shift down by U after each group) or
    // those slots mod Q (U = Q: no shifts).
    {
      const int nseg = zb - za;
      int i = 0;
      while (true) {
#pragma unroll
        for (int ph = 0; ph < U; ++ph) {
          if (i >= nseg) goto segment_done;
          {
            const int zc = za + i;
            const uint32_t slot = su % DU;
            if (!mbar_wait(&full_u[slot], (su / DU) & 1)) goto timeout;
            const float *pl = ring_u + slot * USLOT + (R + row0) * BW + HXB + lane;
#pragma unroll
            for (int h = 0; h < NY / 2; ++h)
              qp[h][tma_qslot<U, Q>(ph, 2 * R)] = make_float2(pl[2 * h * BW], pl[(2 * h + 1) * BW]);
            const uint32_t cs = (su - R) % DU;  // ring-U slot holding plane zc
            const float *cp = ring_u + cs * USLOT + row0 * BW + HXB + lane;
            const float *xs = nullptr;
            uint32_t xslot = 0;
            if (AC) {
              xslot = sx % DX;
              if (!mbar_wait(&full_x[xslot], (sx / DX) & 1)) goto timeout;
              xs = ring_x + xslot * XN * XT + row0 * kTmaTX + lane;
            }
            const bool cone = kUnitC && ucf && ucf[(int64_t)tile * n0 + zc];
            float ycol[NY + 2 * R];  // this thread's column, rows row0-R .. row0+NY-1+R
            // the thread's own rows of plane zc are in its z-queue already (loaded
            // from the same shared-memory words): only the 2R halo rows are read
#pragma unroll
            for (int r = 0; r < NY + 2 * R; ++r) {
              if (r >= R && r < R + NY) {
                const float2 q2 = qp[(r - R) >> 1][tma_qslot<U, Q>(ph, R)];
                ycol[r] = ((r - R) & 1) ? q2.y : q2.x;
              } else {
                ycol[r] = cp[r * BW];
              }
            }
            float val[NY];
            // y-neighbours at ±k of the row pair (j, j+1).  Where R + j + k is even
            // the operands are the column's aligned register pairs and one packed
            // add sums them; otherwise they straddle two pairs and two scalar adds
            // (the same round-to-nearest results) avoid moving them into pairs.
            auto ysum = [&](int j, int k) -> float2 {
              if (((R + j + k) & 1) == 0)
                return __fadd2_rn(make_float2(ycol[R + j + k], ycol[R + j + 1 + k]),
                                  make_float2(ycol[R + j - k], ycol[R + j + 1 - k]));
              return make_float2(__fadd_rn(ycol[R + j + k], ycol[R + j - k]),
                                 __fadd_rn(ycol[R + j + 1 + k], ycol[R + j + 1 - k]));
            };
#pragma unroll
            for (int h = 0; h < NY / 2; ++h) {
              // rows j and j+1 in packed FP32x2 arithmetic (each lane the scalar
              // operation sequence, round to nearest, nothing fused beyond it)
              const int j = 2 * h;
              const float *r0 = cp + (R + j) * BW, *r1 = r0 + BW;
              const float2 uc = qp[h][tma_qslot<U, Q>(ph, R)];
              float2 lo = make_float2(0.f, 0.f), le = lo;
              if (ISO) {
                const float2 nuc6 = __fmul2_rn(make_float2(-6.f, -6.f), uc);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                  const float2 sx =
                      __fadd2_rn(make_float2(r0[k], r1[k]), make_float2(r0[-k], r1[-k]));
                  const float2 sy = ysum(j, k);
                  const float2 sz = __fadd2_rn(qp[h][tma_qslot<U, Q>(ph, R + k)],
                                               qp[h][tma_qslot<U, Q>(ph, R - k)]);
                  const float2 dd = __fadd2_rn(__fadd2_rn(__fadd2_rn(sx, sy), sz), nuc6);
                  const float2 w = weight(2, k);
                  if ((k & 1) || !kSplit)
                    lo = __ffma2_rn(w, dd, lo);
                  else
                    le = __ffma2_rn(w, dd, le);
                }
              } else {
                const float2 nuc2 = __fmul2_rn(make_float2(-2.f, -2.f), uc);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                  float2 acc = ((k & 1) || !kSplit) ? lo : le;
                  acc = __ffma2_rn(
                      weight(2, k),
                      __fadd2_rn(__fadd2_rn(make_float2(r0[k], r1[k]), make_float2(r0[-k], r1[-k])),
                                 nuc2),
                      acc);
                  acc = __ffma2_rn(
                      weight(1, k),
                      __fadd2_rn(ysum(j, k), nuc2),
                      acc);
                  acc = __ffma2_rn(weight(0, k),
                                   __fadd2_rn(__fadd2_rn(qp[h][tma_qslot<U, Q>(ph, R + k)],
                                                         qp[h][tma_qslot<U, Q>(ph, R - k)]),
                                              nuc2),
                                   acc);
                  if ((k & 1) || !kSplit)
                    lo = acc;
                  else
                    le = acc;
                }
              }
              const float2 lap = kSplit ? __fadd2_rn(lo, le) : lo;
              if (AC) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                  const float up = xs[(j + i) * kTmaTX], a = xs[XT + (j + i) * kTmaTX],
                              cc = cone ? 1.f : xs[2 * XT + (j + i) * kTmaTX];
                  const float u = i ? uc.y : uc.x, l = i ? lap.y : lap.x;
                  val[j + i] = fmaf(a, l, fmaf(1.f + cc, u, -cc * up));
                }
              } else {
                const float2 v = __fadd2_rn(uc, lap);
                val[j] = v.x;
                val[j + 1] = v.y;
              }
            }
            if (AC && nxt_z == zc) {
              // source corners at this tile-plane (most planes have none)
              float4 v = make_float4(val[0], 0.f, 0.f, 0.f);
              if constexpr (NY > 1) v.y = val[1];
              if constexpr (NY > 2) v.z = val[2];
              if constexpr (NY > 3) v.w = val[3];
              const SourceHits h =
                  R > 4 ? source_hits_call(sp.entries, sp.src_scale, sp.wav, sp.nsrc, sp.nc, ecur,
                                           eend, zc, ybase, NY, x, lane, nstep, v)
                        : source_hits(sp.entries, sp.src_scale, sp.wav, sp.nsrc, sp.nc, ecur, eend,
                                      zc, ybase, NY, x, lane, nstep, v);
              val[0] = h.v.x;
              if constexpr (NY > 1) val[1] = h.v.y;
              if constexpr (NY > 2) val[2] = h.v.z;
              if constexpr (NY > 3) val[3] = h.v.w;
              ecur = h.ecur;
              nxt_z = h.nxt_z;
            }
#pragma unroll
            for (int j = 0; j < NY; ++j) {
              if (AC) {
                if (rows_ok & (1u << j)) {
                  __stcs(optr + j * g.px, val[j]);  // streaming: not re-read by this launch
                  if constexpr (FWI) {
                    // second time difference for the imaging condition, in the
                    // order the standalone imaging kernel uses
                    const int64_t off = (optr - out) + (int64_t)j * g.px;
                    if (args.d2) {
                      const float2 q2 = qp[j >> 1][tma_qslot<U, Q>(ph, R)];
                      const float uc = (j & 1) ? q2.y : q2.x, up = xs[j * kTmaTX];
                      args.d2[off] = (val[j] - uc) - (uc - up);
                    }
                    if (img)  // img_d2 and the old img from ring X
                      args.img[off] = fmaf(args.img_scale * val[j], xs[3 * XT + j * kTmaTX],
                                           xs[4 * XT + j * kTmaTX]);
                  }
                }
              } else {
                if ((rows_ok & (1u << j)) && (!g.hold || (zc > 0 && zc < n0 - 1)))
                  __stcs(optr + j * g.px, val[j]);
              }
            }
            optr += g.plane;
            __syncwarp();
            if (lane == 0) {
              if (AC) mbar_arrive(&empty_x[xslot]);
              mbar_arrive(&empty_u[cs]);
              if (zc + R >= zb) mbar_arrive(&empty_u[slot]);  // trailing plane: queue only
            }
            if (AC) ++sx;
            ++su;
            ++i;
          }
        }
        if constexpr (U < Q) {
          // slide the window: slots U .. U+2R-1 become 0 .. 2R-1
#pragma unroll
          for (int h = 0; h < NY / 2; ++h)
#pragma unroll
            for (int m = 0; m < 2 * R; ++m) qp[h][m] = qp[h][m + U];
        }
      }
    }
  segment_done:;
  }
  return;
timeout:
  if (lane == 0) {
    if (atomicCAS(err, 0, 1) == 0) err[1] = blockIdx.x;
    *abort_flag = 1;
  }
}

// ---------------------------------------------------------------------------
// Step with two adjacent x points per lane (tiles kXpTX = 64 wide).  Same
// pipeline as k_stencil3d_tma (producer warp, ring U of halo'd u^n planes, ring
// X of (u^{n-1}, A, C) tiles for the acoustic step, register z-queue, whole-
// segment or equal-range split, fused source injection, skip_c), but a consumer
// lane owns the x pair (x0 + 2·lane, x0 + 2·lane + 1) of NY rows: every
// shared-memory read is an 8-byte pair, so a point needs about 5 neighbour reads
// instead of 12 (radius 4), and the packed FP32x2 arithmetic runs over the x
// pair.  The per-point operation sequence is that of k_stencil3d_tma (the same
// sums in the same order, round to nearest; sources added in entry order), so
// results are bitwise the same.  No batched or FWI instances.
//
// QUEUE: instead of a static share of the segments, the CTAs take {0, tile, za,
// zb} items from a work queue (TmaArgs items/wq): z-layers thick first and thin
// last, layer by layer, tile by tile, so the items in flight are neighbouring
// tiles at about the same depth (their halo rows are read from DRAM once) and the
// CTAs finish together.  The producer publishes each item to the consumers in a
// shared-memory ring before the item's first plane; the last CTA out resets the
// queue.  A separate instance, so that the static splits keep their own code.
// ---------------------------------------------------------------------------
constexpr int kXpTX = 64;
// Work-queue items published ahead of use (shared memory at byte 512).  The
// producer writes entry k + kItemRing after issuing every fill of items k ..
// k + kItemRing - 1 (at least 1 + 2R each), which needs the ring-U slot of a
// fill more than a ring depth later to be released: the consumers have read
// entry k by then (static_assert in the kernel).
constexpr int kItemRing = 16;
__host__ __device__ constexpr int xp_bw(int R) { return kXpTX + 2 * tma_hxb(R); }
__host__ __device__ constexpr int xp_ubytes(int R, int NY) { return xp_bw(R) * tma_bh(R, NY) * 4; }
__host__ __device__ constexpr int xp_xbytes(int NY) { return kXpTX * tma_ty(NY) * 4; }
__host__ __device__ constexpr int xp_smem_bytes(int R, int NY, bool acoustic) {
  return 1024 + tma_du(R, acoustic, xp_ubytes(R, NY)) * tma_align128(xp_ubytes(R, NY)) +
         (acoustic ? kTmaDX * 3 * xp_xbytes(NY) : 0);
}
// the queue holds 2·NY·(2R+1) floats a thread
__host__ __device__ constexpr int xp_minb(int R, int NY) { return tma_minb(R, 2 * NY); }
// Tile heights of the x-pair kernel, by height code hc = tile_y / 8 (the host's
// "ny"): 16 rows = 8 consumer warps × 2 rows, 32 = 8 × 4, and 24 = 12 warps × 2
// rows (radius 4 and up: more warps to hide latency where a thread's registers
// allow only one CTA per SM).  The size helpers above take hc.
__host__ __device__ constexpr int xp_nw(int hc) { return hc == 3 ? 12 : kTmaNW; }
__host__ __device__ constexpr int xp_rows(int hc) { return hc == 3 ? 2 : hc; }
__host__ __device__ constexpr bool xp_hc_supported(int R, int hc) {
  return hc == 2 || hc == 4 || (hc == 3 && R >= 4);
}

// Source corners at plane zc of this tile for the lane's x pair: vx holds rows
// 0..3 at x, vy rows 0..3 at x + 1 (see source_hits).
struct SourceHitsXp {
  float4 vx, vy;
  int ecur, nxt_z;
};
__device__ __forceinline__ void add_row(float4 &v, int j, float a) {
  if (j == 0) v.x += a;
  else if (j == 1) v.y += a;
  else if (j == 2) v.z += a;
  else v.w += a;
}
__device__ __forceinline__ SourceHitsXp source_hits_xp(const int4 *entries, const float *src_scale,
                                                       const float *wav, int nsrc, int nc,
                                                       int ecur, int eend, int zc, int ybase,
                                                       int ny, int x, int lane, int64_t nstep,
                                                       float4 vx, float4 vy) {
  while (true) {
    const int e = ecur + lane;
    const int4 en = e < eend ? entries[e] : make_int4(0, 0, INT_MAX, 0);
    const int cnt = __popc(__ballot_sync(0xffffffffu, en.z == zc));  // a prefix
    const int jr = en.y - ybase;
    const bool here = en.z == zc && jr >= 0 && jr < ny;
    float add = 0.f;
    if (here) add = src_scale[en.w] * wav[nstep * nsrc + en.w / nc];
    unsigned mine = __ballot_sync(0xffffffffu, here);
    while (mine) {
      const int b = __ffs(mine) - 1;
      mine &= mine - 1;
      const int ex = __shfl_sync(0xffffffffu, en.x, b);
      const int ej = __shfl_sync(0xffffffffu, jr, b);
      const float ad = __shfl_sync(0xffffffffu, add, b);
      if (ex == x) add_row(vx, ej, ad);
      else if (ex == x + 1) add_row(vy, ej, ad);
    }
    ecur += cnt;
    if (cnt < 32) break;
  }
  SourceHitsXp h;
  h.vx = vx;
  h.vy = vy;
  h.ecur = ecur;
  h.nxt_z = ecur < eend ? entries[ecur].z : INT_MAX;
  return h;
}
__device__ __noinline__ SourceHitsXp source_hits_xp_call(const int4 *entries,
                                                         const float *src_scale, const float *wav,
                                                         int nsrc, int nc, int ecur, int eend,
                                                         int zc, int ybase, int ny, int x,
                                                         int lane, int64_t nstep, float4 vx,
                                                         float4 vy) {
  return source_hits_xp(entries, src_scale, wav, nsrc, nc, ecur, eend, zc, ybase, ny, x, lane,
                        nstep, vx, vy);
}

template <int R, int NY, int EQ, bool ISO, bool QUEUE = false, int NW = kTmaNW>
__global__ void __launch_bounds__((NW + 1) * 32, NW == kTmaNW ? xp_minb(R, NY) : 1)
k_stencil3d_xp(const __grid_constant__ CUtensorMap map_u,  // u^n, halo box (kXpTX + 2·HXB wide)
               const __grid_constant__ CUtensorMap map_p,  // u^{n-1}, tile box (kXpTX wide)
               const __grid_constant__ CUtensorMap map_a,  // A, tile box
               const __grid_constant__ CUtensorMap map_c,  // C, tile box
               const __grid_constant__ CUtensorMap, const __grid_constant__ CUtensorMap,
               const TmaArgs args, const BatchArgs) {
  constexpr bool AC = EQ == kAcoustic;
  constexpr int HC = NW * NY / kTmaNW;                       // height code (tile_y / 8)
  static_assert(NW * NY % kTmaNW == 0 && xp_nw(HC) == NW && xp_rows(HC) == NY, "tile shape");
  constexpr int TY = tma_ty(HC);                               // NW·NY rows
  constexpr int HXB = tma_hxb(R), BW = xp_bw(R), DU = tma_du(R, AC, xp_ubytes(R, HC)), DX = kTmaDX;
  constexpr int USLOT = tma_align128(xp_ubytes(R, HC)) / 4;  // floats per ring-U slot
  constexpr int XT = kXpTX * TY;                              // floats per ring-X tile
  constexpr int Q = 2 * R + 1;
  // 12 consumer warps run at the 128-register cap of 416 threads: the acoustic step
  // unrolls by 2 there (two fewer queue planes a row, no spills; so 16 at 512³ 542 ->
  // 533 µs) where the window is not unrolled whole; diffusion lost 3-4 % that way
  constexpr int U = (EQ == kAcoustic && NW != kTmaNW && tma_unroll(R) < 2 * R + 1)
                        ? 2
                        : tma_unroll(R);
  constexpr int QL = U == Q ? Q : Q + U - 1;
  constexpr bool kSplit = R > 4;
  constexpr bool kUnitC = AC && R <= 4;
  constexpr int PH = (R + 1) / 2;  // x pairs each side of the lane's own
  static_assert(NY <= 4, "source rows are carried in a float4");
  static_assert(!QUEUE || ((2 * DU + 2 * DX) * 8 + 4 <= 512 &&
                           kItemRing * (1 + 2 * R) >= DU + 1 && 512 + kItemRing * 16 <= 1024),
                "item ring: overlaps the barriers, or too shallow for ring U");
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *full_u = reinterpret_cast<uint64_t *>(smem);
  uint64_t *empty_u = full_u + DU;
  uint64_t *full_x = empty_u + DU;
  uint64_t *empty_x = full_x + DX;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty_x + DX);
  volatile int4 *item_ring = reinterpret_cast<volatile int4 *>(smem + 512);  // QUEUE only
  float *ring_u = reinterpret_cast<float *>(smem + 1024);
  float *ring_x = ring_u + DU * USLOT;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int *const err = args.err;
  if (threadIdx.x == 0) {
    for (int i = 0; i < DU; ++i) {
      mbar_init(&full_u[i], 1);
      mbar_init(&empty_u[i], NW);
    }
    for (int i = 0; i < DX; ++i) {
      mbar_init(&full_x[i], 1);
      mbar_init(&empty_x[i], NW);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  int64_t q0 = 0, q1 = 0;
  if constexpr (!QUEUE) {
    if (args.aligned)
      cta_range((int64_t)args.ntiles * ((args.g.n0 + args.zblock - 1) / args.zblock), blockIdx.x,
                gridDim.x, q0, q1);
    else
      cta_range(args.W, blockIdx.x, gridDim.x, q0, q1);
  }
  const unsigned char *ucf = kUnitC ? args.unit_c : nullptr;

  if (warp == NW) {
    // ------------------------------- producer -------------------------------
    if (lane == 0) {
      tma_prefetch_desc(&map_u);
      if (AC) {
        tma_prefetch_desc(&map_p);
        tma_prefetch_desc(&map_a);
        tma_prefetch_desc(&map_c);
      }
      uint32_t su = 0, sx = 0;
      const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
      bool ok = true;
      int64_t q = q0;
      unsigned nitem = 0;  // QUEUE: items taken by this block
      while (ok && (QUEUE || q < q1)) {
        int tile, za, zb;
        if constexpr (QUEUE) {
          const int4 item = take_item(args.wq, args.items, args.nitems);
          item_ring[nitem % kItemRing].x = item.x;
          item_ring[nitem % kItemRing].y = item.y;
          item_ring[nitem % kItemRing].z = item.z;
          item_ring[nitem % kItemRing].w = item.w;
          ++nitem;
          if (item.x < 0) {
            // no work left: complete the next ring-U phase without data so the
            // consumers read the end mark published above
            const uint32_t slot = su % DU;
            if (su >= (uint32_t)DU && !mbar_wait(&empty_u[slot], ((su / DU) - 1) & 1)) {
              ok = false;
              break;
            }
            mbar_arrive(&full_u[slot]);
            ++su;
            break;
          }
          tile = item.y;
          za = item.z;
          zb = item.w;
        } else {
          next_segment(args, q, q1, tile, za, zb);
        }
        const int x0 = (tile % args.tiles_x) * kXpTX, y0 = (tile / args.tiles_x) * TY;
        for (int p = za - R; p < zb + R; ++p) {
          if (*abort_flag) { ok = false; break; }
          const int zc = p - R;
          if (AC && zc >= za) {
            const uint32_t slot = sx % DX;
            if (sx >= (uint32_t)DX && !mbar_wait(&empty_x[slot], ((sx / DX) - 1) & 1)) {
              ok = false;
              break;
            }
            float *dst = ring_x + slot * 3 * XT;
            const bool cone = kUnitC && ucf && ucf[(int64_t)tile * args.g.n0 + zc];
            mbar_expect_tx(&full_x[slot], (3 - (cone ? 1 : 0)) * XT * 4);
            const MapOrigin &o = args.org;
            const int tx = x0 + o.ox, ty = y0 + o.oy, tz = zc + o.oz;  // tile box
            tma_load_3d_hint(dst, &map_p, tx, ty, tz, &full_x[slot], once);
            tma_load_3d_hint(dst + XT, &map_a, tx, ty, tz, &full_x[slot], once);
            if (!cone) tma_load_3d_hint(dst + 2 * XT, &map_c, tx, ty, tz, &full_x[slot], once);
            ++sx;
          }
          const uint32_t slot = su % DU;
          if (su >= (uint32_t)DU && !mbar_wait(&empty_u[slot], ((su / DU) - 1) & 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full_u[slot], xp_ubytes(R, HC));
          tma_load_3d_hint(ring_u + slot * USLOT, &map_u, x0 - HXB + args.org.ox,
                           y0 - R + args.org.oy, p + args.org.oz, &full_u[slot], keep);
          ++su;
        }
      }
      if (!ok && atomicCAS(err, 0, 2) == 0) err[1] = blockIdx.x;
      if (!ok) *abort_flag = 1;
      bool drained = true;
      for (uint32_t i = 0; i < (uint32_t)DU && i < su; ++i) {
        const uint32_t last = su - 1 - ((su - 1 - i) % DU);  // last fill of slot i
        drained &= mbar_wait(&full_u[last % DU], (last / DU) & 1);
      }
      for (uint32_t i = 0; i < (uint32_t)DX && i < sx; ++i) {
        const uint32_t last = sx - 1 - ((sx - 1 - i) % DX);
        drained &= mbar_wait(&full_x[last % DX], (last / DX) & 1);
      }
      if (!drained && atomicCAS(err, 0, 3) == 0) err[1] = blockIdx.x;
      if constexpr (QUEUE) queue_done(args.wq);
    }
    return;
  }

  // --------------------------------- consumers --------------------------------
  float2 qp[NY][QL];  // queue: row j, the lane's x pair
  // ring-U position of the next fill to consume: slot and phase parity, kept
  // incrementally (DU is not a power of two; no division per plane)
  uint32_t uslot = 0, upar = 0, sx = 0;
  auto next_u = [&]() {
    if (++uslot == (uint32_t)DU) {
      uslot = 0;
      upar ^= 1u;
    }
  };
  const int row0 = warp * NY;
  const float2 *wp0 = args.c.wp[0], *wp1 = args.c.wp[1], *wp2 = args.c.wp[2];
  const Geom g = args.g;
  const SparseArgs sp = args.sp;
  const int64_t nstep = (AC && sp.step) ? *sp.step + sp.j : 0;
  float *const out = args.out;
  int64_t q = q0;
  unsigned nitem = 0;
  while (QUEUE || q < q1) {
    int tile, za, zb;
    if constexpr (QUEUE) {
      // the next item is published with the first fill of its planes
      if (!mbar_wait(&full_u[uslot], upar)) goto timeout;
      const int4 item = make_int4(item_ring[nitem % kItemRing].x, item_ring[nitem % kItemRing].y,
                                  item_ring[nitem % kItemRing].z, item_ring[nitem % kItemRing].w);
      ++nitem;
      if (item.x < 0) break;
      tile = item.y;
      za = item.z;
      zb = item.w;
    } else {
      next_segment(args, q, q1, tile, za, zb);
    }
    const int n0 = g.n0;
    const int x = (tile % args.tiles_x) * kXpTX + 2 * lane;
    const int ybase = (tile / args.tiles_x) * TY + row0;
    // which of the pair's points a row stores: acoustic every node, diffusion
    // interior nodes only (every node without the held boundary)
    const bool all = AC || !g.hold;
    const bool xin0 = all ? x < g.n2 : (x > 0 && x < g.n2 - 1);
    const bool xin1 = all ? x + 1 < g.n2 : (x + 1 > 0 && x + 1 < g.n2 - 1);
    unsigned rows_ok = 0;
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      const int y = ybase + j;
      rows_ok |= ((all ? y < g.n1 : (y > 0 && y < g.n1 - 1)) ? 1u : 0u) << j;
    }
    float *optr = out + gidx(g, za, ybase, x);
    int ecur = 0, eend = 0, nxt_z = INT_MAX;
    if (AC && sp.first) {
      ecur = sp.first[tile * n0 + za];
      eend = sp.first[tile * n0 + zb];
      if (ecur < eend) nxt_z = sp.entries[ecur].z;
    }
    // warm-up: planes za-R .. za+R-1 fill queue slots 0 .. 2R-1
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) {
      const int p = za - R + m;
      const uint32_t slot = uslot;
      if (!mbar_wait(&full_u[slot], upar)) goto timeout;
      const float *pl = ring_u + slot * USLOT + (R + row0) * BW + HXB + 2 * lane;
#pragma unroll
      for (int j = 0; j < NY; ++j) qp[j][m] = *reinterpret_cast<const float2 *>(pl + j * BW);
      if (p < za || p >= zb) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_u[slot]);
      }
      next_u();
    }
    {
      const int nseg = zb - za;
      int i = 0;
      while (true) {
#pragma unroll
        for (int ph = 0; ph < U; ++ph) {
          if (i >= nseg) goto segment_done;
          {
            const int zc = za + i;
            const uint32_t slot = uslot;
            if (!mbar_wait(&full_u[slot], upar)) goto timeout;
            const float *pl = ring_u + slot * USLOT + (R + row0) * BW + HXB + 2 * lane;
#pragma unroll
            for (int j = 0; j < NY; ++j)
              qp[j][tma_qslot<U, Q>(ph, 2 * R)] = *reinterpret_cast<const float2 *>(pl + j * BW);
            // ring-U slot holding plane zc, R fills back (at least 2R fills consumed)
            const uint32_t cs = slot >= (uint32_t)R ? slot - R : slot + DU - R;
            const float *cp = ring_u + cs * USLOT + row0 * BW + HXB + 2 * lane;
            const float *xs = nullptr;
            uint32_t xslot = 0;
            if (AC) {
              xslot = sx % DX;
              if (!mbar_wait(&full_x[xslot], (sx / DX) & 1)) goto timeout;
              xs = ring_x + xslot * 3 * XT + row0 * kXpTX + 2 * lane;
            }
            const bool cone = kUnitC && ucf && ucf[(int64_t)tile * n0 + zc];
            float2 ycol[NY + 2 * R];  // the lane's pair, rows row0-R .. row0+NY-1+R
            // the thread's own rows of plane zc are in its z-queue already (loaded
            // from the same shared-memory words): only the 2R halo rows are read
#pragma unroll
            for (int r = 0; r < NY + 2 * R; ++r)
              ycol[r] = (r >= R && r < R + NY) ? qp[r - R][tma_qslot<U, Q>(ph, R)]
                                               : *reinterpret_cast<const float2 *>(cp + r * BW);
            float2 val[NY];
#pragma unroll
            for (int j = 0; j < NY; ++j) {
              // the row's x pairs around the lane's own (pair d starts at x + 2d)
              const float *rp = cp + (R + j) * BW;
              float2 xpr[2 * PH + 1];
#pragma unroll
              for (int d = -PH; d <= PH; ++d)
                xpr[d + PH] = d == 0 ? ycol[R + j] : *reinterpret_cast<const float2 *>(rp + 2 * d);
              // u(x+k) + u(x-k) for the pair: aligned pairs for even k, halves of
              // the neighbouring pairs for odd k
              auto xsum = [&](int k) -> float2 {
                if ((k & 1) == 0) return __fadd2_rn(xpr[PH + k / 2], xpr[PH - k / 2]);
                return make_float2(__fadd_rn(xpr[PH + (k - 1) / 2].y, xpr[PH - (k + 1) / 2].y),
                                   __fadd_rn(xpr[PH + (k + 1) / 2].x, xpr[PH - (k - 1) / 2].x));
              };
              const float2 uc = qp[j][tma_qslot<U, Q>(ph, R)];
              float2 lo = make_float2(0.f, 0.f), le = lo;
              if (ISO) {
                const float2 nuc6 = __fmul2_rn(make_float2(-6.f, -6.f), uc);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                  const float2 sx2 = xsum(k);
                  const float2 sy = __fadd2_rn(ycol[R + j + k], ycol[R + j - k]);
                  const float2 sz = __fadd2_rn(qp[j][tma_qslot<U, Q>(ph, R + k)],
                                               qp[j][tma_qslot<U, Q>(ph, R - k)]);
                  const float2 dd = __fadd2_rn(__fadd2_rn(__fadd2_rn(sx2, sy), sz), nuc6);
                  if ((k & 1) || !kSplit)
                    lo = __ffma2_rn(wp2[k], dd, lo);
                  else
                    le = __ffma2_rn(wp2[k], dd, le);
                }
              } else {
                const float2 nuc2 = __fmul2_rn(make_float2(-2.f, -2.f), uc);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                  float2 acc = ((k & 1) || !kSplit) ? lo : le;
                  acc = __ffma2_rn(wp2[k], __fadd2_rn(xsum(k), nuc2), acc);
                  acc = __ffma2_rn(wp1[k],
                                   __fadd2_rn(__fadd2_rn(ycol[R + j + k], ycol[R + j - k]), nuc2),
                                   acc);
                  acc = __ffma2_rn(wp0[k],
                                   __fadd2_rn(__fadd2_rn(qp[j][tma_qslot<U, Q>(ph, R + k)],
                                                         qp[j][tma_qslot<U, Q>(ph, R - k)]),
                                              nuc2),
                                   acc);
                  if ((k & 1) || !kSplit)
                    lo = acc;
                  else
                    le = acc;
                }
              }
              const float2 lap = kSplit ? __fadd2_rn(lo, le) : lo;
              if (AC) {
                // u^{n+1} = A·lap + (1 + C)·u − C·u^{n−1}, per point as k_stencil3d_tma
                const float2 up = *reinterpret_cast<const float2 *>(xs + j * kXpTX);
                const float2 a = *reinterpret_cast<const float2 *>(xs + XT + j * kXpTX);
                const float2 cc = cone ? make_float2(1.f, 1.f)
                                       : *reinterpret_cast<const float2 *>(xs + 2 * XT + j * kXpTX);
                val[j].x = fmaf(a.x, lap.x, fmaf(1.f + cc.x, uc.x, -cc.x * up.x));
                val[j].y = fmaf(a.y, lap.y, fmaf(1.f + cc.y, uc.y, -cc.y * up.y));
              } else {
                val[j] = __fadd2_rn(uc, lap);
              }
            }
            if (AC && nxt_z == zc) {
              // source corners at this tile-plane (most planes have none)
              float4 vx = make_float4(val[0].x, 0.f, 0.f, 0.f), vy = make_float4(val[0].y, 0.f, 0.f, 0.f);
              if constexpr (NY > 1) { vx.y = val[1].x; vy.y = val[1].y; }
              if constexpr (NY > 2) { vx.z = val[2].x; vy.z = val[2].y; }
              if constexpr (NY > 3) { vx.w = val[3].x; vy.w = val[3].y; }
              const SourceHitsXp h =
                  R > 4 ? source_hits_xp_call(sp.entries, sp.src_scale, sp.wav, sp.nsrc, sp.nc,
                                              ecur, eend, zc, ybase, NY, x, lane, nstep, vx, vy)
                        : source_hits_xp(sp.entries, sp.src_scale, sp.wav, sp.nsrc, sp.nc, ecur,
                                         eend, zc, ybase, NY, x, lane, nstep, vx, vy);
              val[0] = make_float2(h.vx.x, h.vy.x);
              if constexpr (NY > 1) val[1] = make_float2(h.vx.y, h.vy.y);
              if constexpr (NY > 2) val[2] = make_float2(h.vx.z, h.vy.z);
              if constexpr (NY > 3) val[3] = make_float2(h.vx.w, h.vy.w);
              ecur = h.ecur;
              nxt_z = h.nxt_z;
            }
            // diffusion: interior planes only (boundary values stay as set)
            if (all || (zc > 0 && zc < n0 - 1)) {
#pragma unroll
              for (int j = 0; j < NY; ++j) {
                if (!(rows_ok & (1u << j))) continue;
                float *o = optr + j * g.px;
                if (xin0 && xin1)
                  __stcs(reinterpret_cast<float2 *>(o), val[j]);
                else {
                  if (xin0) __stcs(o, val[j].x);
                  if (xin1) __stcs(o + 1, val[j].y);
                }
              }
            }
            optr += g.plane;
            __syncwarp();
            if (lane == 0) {
              if (AC) mbar_arrive(&empty_x[xslot]);
              mbar_arrive(&empty_u[cs]);
              if (zc + R >= zb) mbar_arrive(&empty_u[slot]);  // trailing plane: queue only
            }
            if (AC) ++sx;
            next_u();
            ++i;
          }
        }
        if constexpr (U < Q) {
#pragma unroll
          for (int j = 0; j < NY; ++j)
#pragma unroll
            for (int m = 0; m < 2 * R; ++m) qp[j][m] = qp[j][m + U];
        }
      }
    }
  segment_done:;
  }
  return;
timeout:
  if (lane == 0) {
    if (atomicCAS(err, 0, 1) == 0) err[1] = blockIdx.x;
    *abort_flag = 1;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using TmaKernelFn = void (*)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap,
                             CUtensorMap, TmaArgs, BatchArgs);

struct TmaPlan {
  const char *name = "none";
  CUtensorMap map_u[2];   // u levels, halo box
  CUtensorMap map_t[2];   // u levels, tile box (u^{n-1} reads)
  CUtensorMap map_a, map_c;
  TmaArgs args{};
  float *level[2] = {nullptr, nullptr};
  TmaKernelFn fn = nullptr;        // one shot, tile height 8·ny
  TmaKernelFn fn_multi = nullptr;  // batches (default tile height only)
  TmaKernelFn fn_fwi = nullptr;    // one shot with the FWI epilogue (acoustic)
  int grid = 0, smem = 0;
  int threads = kTmaThreads;  // of fn: (consumer warps + 1) × 32
  int grid_multi = 0, smem_multi = 0;
  int ny = 0;          // rows per consumer thread
  int per_sm = 0;      // resident CTAs per SM the persistent grid is sized for
  int per_sm_max = 0;  // occupancy limit of fn
  int per_sm_fwi = 0;  // occupancy limit of fn_fwi
  int smem_fwi = 0;
  int sms = 0;
  int tx = kTmaTX;     // tile width: kTmaTX, or kXpTX (two x points a lane)
  // work queue (aligned = 2): device memory {ticket, done, 0, 0} followed by the
  // items; shared by the copies of this plan, freed with the last
  std::shared_ptr<int4> wq_mem;
  std::vector<int> layers;  // the queue's z-layer heights, thick first
};

// Z-layer heights of a work queue of ntiles tiles over n0 planes for G CTAs.
// Items are taken in order (layer by layer, tile by tile) by whichever CTA is
// free, so the layers are thick while much work remains and thinner towards the
// end: each layer about the remaining work per CTA over f, none thinner than
// hmin (hcap > 0: none thicker than hcap).  Among f in {1, 1.5, 2, 3} and hmin in
// {8, max(8, 2R)} the one with the shortest predicted makespan wins (list
// scheduling of the items in order; an item of h planes costs h plus 0.3 per halo
// plane it streams, 2R of them).
inline std::vector<int> queue_layers(int n0, int ntiles, int G, int R, int hcap) {
  auto build = [&](double f, int hmin) {
    std::vector<int> hs;
    hmin = std::min(hmin, n0);
    for (int z = 0; z < n0;) {
      const int rem = n0 - z;
      int64_t h = (int64_t)std::ceil((double)rem * ntiles / (f * G));
      h = std::max<int64_t>(h, hmin);
      if (hcap > 0) h = std::min<int64_t>(h, std::max(hcap, hmin));
      h = std::min<int64_t>(h, rem);
      if (rem - h < hmin) h = rem;
      hs.push_back((int)h);
      z += (int)h;
    }
    return hs;
  };
  auto makespan = [&](const std::vector<int> &hs) {
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int i = 0; i < G; ++i) free_at.push(0.0);
    double end = 0.0;
    for (int h : hs)
      for (int t = 0; t < ntiles; ++t) {
        const double t1 = free_at.top() + h + 0.3 * 2 * R;
        free_at.pop();
        end = std::max(end, t1);
        free_at.push(t1);
      }
    return end;
  };
  std::vector<int> best;
  double best_t = 1e300;
  for (double f : {1.0, 1.5, 2.0, 3.0})
    for (int hmin : {8, std::max(8, 2 * R)}) {
      std::vector<int> hs = build(f, hmin);
      const double t = makespan(hs);
      if (t < best_t - 1e-9) {
        best_t = t;
        best = hs;
      }
    }
  return best;
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

inline EncodeFn tma_encoder() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}

// A map of one padded field (base = its first padded element) with coordinate 0
// of each axis at the origin o (see MapOrigin): an interior axis spans the n
// interior nodes, a padded one the whole padded extent.
inline bool encode_map(EncodeFn enc, CUtensorMap *m, float *field, const Geom &g, int bw, int bh,
                       const MapOrigin &o) {
  float *base = field + (int64_t)(g.R0 - o.oz) * g.plane + (int64_t)(g.R - o.oy) * g.px +
                (kHaloX - o.ox);
  const cuuint64_t dims[3] = {(cuuint64_t)(o.ox ? g.px : g.n2), (cuuint64_t)(o.oy ? g.py : g.n1),
                              (cuuint64_t)(o.oz ? g.n0 + 2 * g.R0 : g.n0)};
  const cuuint64_t strides[2] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int R, int NY, int EQ, bool ISO, bool MULTI, bool FWI = false>
inline cudaError_t tma_instance(TmaKernelFn &fn, int &smem, int &per_sm) {
  fn = k_stencil3d_tma<R, NY, EQ, ISO, MULTI, FWI>;
  smem = tma_smem_bytes(R, NY, EQ == kAcoustic, FWI);
  cudaError_t e = cudaFuncSetAttribute(k_stencil3d_tma<R, NY, EQ, ISO, MULTI, FWI>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, k_stencil3d_tma<R, NY, EQ, ISO, MULTI, FWI>, kTmaThreads, smem);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  return e;
}

// Kernel instances for rows-per-thread ny (2 or 4); batches use the default.
template <int R, int EQ, bool ISO>
inline cudaError_t tma_configure(TmaPlan &pl, int ny) {
  constexpr int NYD = tma_ny(R);
  pl.threads = kTmaThreads;
  cudaError_t e = ny == 2 ? tma_instance<R, 2, EQ, ISO, false>(pl.fn, pl.smem, pl.per_sm_max)
                          : tma_instance<R, 4, EQ, ISO, false>(pl.fn, pl.smem, pl.per_sm_max);
  if (e != cudaSuccess) return e;
  pl.fn_multi = nullptr;
  pl.fn_fwi = nullptr;
  pl.smem_multi = 0;
  int per_sm_multi = 0;
  if constexpr (EQ == kAcoustic) {
    e = tma_instance<R, NYD, EQ, ISO, true>(pl.fn_multi, pl.smem_multi, per_sm_multi);
    if (e != cudaSuccess) return e;
    // the FWI epilogue instance of this tile; its occupancy must cover the plan's
    // grid (checked once the grid is known)
    e = ny == 2 ? tma_instance<R, 2, EQ, ISO, false, true>(pl.fn_fwi, pl.smem_fwi, pl.per_sm_fwi)
                : tma_instance<R, 4, EQ, ISO, false, true>(pl.fn_fwi, pl.smem_fwi, pl.per_sm_fwi);
    if (e != cudaSuccess) return e;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&pl.sms, cudaDevAttrMultiProcessorCount, dev);
  pl.grid_multi = pl.sms * std::max(per_sm_multi, 1);
  return cudaSuccess;
}

// The x-pair kernel for rows-per-thread ny.
template <int R, int EQ, bool ISO>
inline cudaError_t xp_configure(TmaPlan &pl, int ny, bool queue) {
  // ny is the height code: 2 → 8 warps × 2 rows, 3 → 12 × 2 (radius 4 and up), 4 → 8 × 4
  TmaKernelFn fn = nullptr;
  if (ny == 2)
    fn = queue ? k_stencil3d_xp<R, 2, EQ, ISO, true> : k_stencil3d_xp<R, 2, EQ, ISO>;
  else if (ny == 4)
    fn = queue ? k_stencil3d_xp<R, 4, EQ, ISO, true> : k_stencil3d_xp<R, 4, EQ, ISO>;
  else if constexpr (xp_hc_supported(R, 3)) {
    if (ny == 3)
      fn = queue ? k_stencil3d_xp<R, 2, EQ, ISO, true, 12> : k_stencil3d_xp<R, 2, EQ, ISO, false, 12>;
  }
  if (!fn) return cudaErrorInvalidValue;
  const int threads = (xp_nw(ny) + 1) * 32;
  const int smem = xp_smem_bytes(R, ny, EQ == kAcoustic);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl.per_sm_max, fn, threads, smem);
  if (e == cudaSuccess && pl.per_sm_max < 1) e = cudaErrorInvalidConfiguration;
  if (e != cudaSuccess) return e;
  pl.fn = fn;
  pl.smem = smem;
  pl.threads = threads;
  pl.fn_multi = nullptr;
  pl.fn_fwi = nullptr;
  pl.smem_multi = 0;
  pl.per_sm_fwi = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&pl.sms, cudaDevAttrMultiProcessorCount, dev);
  pl.grid_multi = 0;
  return cudaSuccess;
}

// Tile configurations the pipelined kernel offers (the autotuner's space).
inline bool tma_ny_supported(int ny) { return ny == 2 || ny == 3 || ny == 4; }
inline bool tma_tx_supported(int tx, int) { return tx == kTmaTX || tx == kXpTX; }

// Build the plan: tensor maps for both levels and the coefficient fields, for
// ny rows per consumer thread (0: the default), a grid of per_sm CTAs per SM
// (0: as many as fit) and z-blocks of zblock planes (0: about one CTA's share).
// Map origin of a context: interior maps (zeros outside the grid from TMA's fill)
// unless the halo holds data: padded in every axis for the odd-reflection
// boundary, padded along z for a z-slab sub-domain (the neighbours' planes).
inline MapOrigin map_origin(const Geom &g, bool odd_halo, bool z_halo) {
  if (odd_halo) return MapOrigin{kHaloX, g.R, g.R0};
  return MapOrigin{0, 0, z_halo ? g.R0 : 0};
}

inline cudaError_t plan_tma(TmaPlan &pl, const Geom &g, int eq, bool iso, float *const *level,
                            float *A, float *C, int ny, int per_sm, int zblock, int aligned,
                            const char **why, int tx = kTmaTX,
                            MapOrigin org = MapOrigin{0, 0, 0}) {
  *why = nullptr;
  if (g.R0 == 0 || g.R < 1 || g.R > kMaxR) {
    *why = "3-D grids only";
    return cudaErrorNotSupported;
  }
  const int R = g.R;
  if (ny == 0) ny = tma_ny(R);
  if (!tma_ny_supported(ny) || !tma_tx_supported(tx, eq) || per_sm < 0 || zblock < 0 ||
      aligned < 0 || aligned > 2 || (aligned == 2 && tx != kXpTX) ||
      (ny == 3 && (tx != kXpTX || !xp_hc_supported(R, 3)))) {
    *why = "unsupported tile configuration";
    return cudaErrorInvalidValue;
  }
  // TMA rules: 16-B aligned bases and strides, inner box extent a 16-B multiple,
  // x coordinates multiples of 4 floats (x0 - HXB + ox with x0 % 32 == 0, ox 0 or kHaloX).
  if ((g.px * 4) % 16 || tma_hxb(R) % 4 || (tma_bw(R) * 4) % 16 || kHaloX % 4 ||
      tma_bw(R) > 256 || tma_bh(R, 4) > 256 || tma_ty(4) > 256 || (kTmaTX * 4) % 16 ||
      (xp_bw(R) * 4) % 16 || xp_bw(R) > 256 || kXpTX % 4) {
    *why = "layout violates the TMA alignment rules";
    return cudaErrorNotSupported;
  }
  EncodeFn enc = tma_encoder();
  if (!enc) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaErrorNotSupported;
  }
  const int ty = tma_ty(ny);
  const bool xp = tx == kXpTX;
  for (int b = 0; b < 2; ++b) {
    if (!encode_map(enc, &pl.map_u[b], level[b], g, xp ? xp_bw(R) : tma_bw(R), tma_bh(R, ny),
                    org) ||
        !encode_map(enc, &pl.map_t[b], level[b], g, tx, ty, org)) {
      *why = "tensor map encoding failed";
      return cudaErrorInvalidValue;
    }
    pl.level[b] = level[b];
  }
  if (eq == kAcoustic) {
    if (!encode_map(enc, &pl.map_a, A, g, tx, ty, org) ||
        !encode_map(enc, &pl.map_c, C, g, tx, ty, org)) {
      *why = "tensor map encoding failed";
      return cudaErrorInvalidValue;
    }
  } else {
    pl.map_a = pl.map_t[0];
    pl.map_c = pl.map_t[0];
  }
  cudaError_t e = cudaErrorNotSupported;
  const bool ac = eq == kAcoustic;
#define TMA_CASE(RR)                                                                   \
  case RR:                                                                             \
    e = ac ? (iso ? tma_configure<RR, kAcoustic, true>(pl, ny)                         \
                  : tma_configure<RR, kAcoustic, false>(pl, ny))                       \
           : (iso ? tma_configure<RR, kDiffusion, true>(pl, ny)                        \
                  : tma_configure<RR, kDiffusion, false>(pl, ny));                     \
    break;
#define XP_CASE(RR)                                                                    \
  case RR:                                                                             \
    e = ac ? (iso ? xp_configure<RR, kAcoustic, true>(pl, ny, aligned == 2)            \
                  : xp_configure<RR, kAcoustic, false>(pl, ny, aligned == 2))          \
           : (iso ? xp_configure<RR, kDiffusion, true>(pl, ny, aligned == 2)           \
                  : xp_configure<RR, kDiffusion, false>(pl, ny, aligned == 2));        \
    break;
  if (xp) {
    switch (R) { XP_CASE(1) XP_CASE(2) XP_CASE(3) XP_CASE(4) XP_CASE(5) XP_CASE(6) XP_CASE(7) XP_CASE(8) }
  } else {
    switch (R) { TMA_CASE(1) TMA_CASE(2) TMA_CASE(3) TMA_CASE(4) TMA_CASE(5) TMA_CASE(6) TMA_CASE(7) TMA_CASE(8) }
  }
#undef XP_CASE
#undef TMA_CASE
  if (e != cudaSuccess) {
    *why = "kernel configuration failed";
    return e;
  }
  if (per_sm > pl.per_sm_max) {
    *why = "more CTAs per SM than fit";
    return cudaErrorInvalidValue;
  }
  pl.ny = ny;
  pl.per_sm = per_sm ? per_sm : pl.per_sm_max;
  pl.grid = pl.sms * pl.per_sm;
  if (pl.fn_fwi && pl.per_sm_fwi < pl.per_sm) pl.fn_fwi = nullptr;  // would not all be resident
  pl.args.g = g;
  pl.args.org = org;
  pl.tx = tx;
  pl.args.tiles_x = (g.n2 + tx - 1) / tx;
  const int tiles_y = (g.n1 + ty - 1) / ty;
  pl.args.ntiles = pl.args.tiles_x * tiles_y;
  pl.args.W = (int64_t)pl.args.ntiles * g.n0;
  pl.args.aligned = aligned;
  pl.args.items = nullptr;
  pl.args.nitems = 0;
  pl.args.wq = nullptr;
  pl.wq_mem.reset();
  pl.layers.clear();
  if (aligned == 2) {
    // work queue: z-layers (zblock > 0 caps their height), items layer by layer
    pl.layers = queue_layers(g.n0, pl.args.ntiles, pl.grid, R, zblock);
    std::vector<int4> h(1, make_int4(0, 0, 0, 0));  // the counters
    int za = 0;
    for (int hk : pl.layers) {
      for (int t = 0; t < pl.args.ntiles; ++t) h.push_back(make_int4(0, t, za, za + hk));
      za += hk;
    }
    int4 *d = nullptr;
    cudaError_t e2 = cudaMalloc(&d, h.size() * sizeof(int4));
    if (e2 == cudaSuccess) {
      pl.wq_mem.reset(d, [](int4 *ptr) { cudaFree(ptr); });
      e2 = cudaMemcpy(d, h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    if (e2 != cudaSuccess) {
      pl.wq_mem.reset();
      *why = "work queue allocation failed";
      return e2;
    }
    pl.args.wq = reinterpret_cast<unsigned *>(d);
    pl.args.items = d + 1;
    pl.args.nitems = (int)(h.size() - 1);
    pl.args.zblock = zblock;  // the cap as given (0: none); the kernel reads the items
    if (pl.grid > pl.args.nitems) pl.grid = pl.args.nitems;
  } else if (aligned) {
    // whole segments: z-blocks of zblock planes (0: as many blocks as make the
    // segments about fill the grid), at most one CTA per segment
    int zb = zblock;
    if (!zb) {  // no segment shorter than max(8, 2R) planes
      const int mcap = std::max(1, g.n0 / std::max(8, 2 * R));
      const int m = std::min(mcap, std::max(1, pl.grid / pl.args.ntiles));
      zb = (g.n0 + m - 1) / m;
    }
    pl.args.zblock = std::min(g.n0, zb);
    const int64_t S = (int64_t)pl.args.ntiles * ((g.n0 + pl.args.zblock - 1) / pl.args.zblock);
    if (pl.grid > S) pl.grid = (int)S;
  } else {
    if (pl.grid > pl.args.W) pl.grid = (int)pl.args.W;
    // z-block height: about one CTA's share, so neighbouring tiles stream in step
    const int64_t share = (pl.args.W + pl.grid - 1) / pl.grid;
    const int64_t zb = zblock ? zblock : std::max<int64_t>(1, share);
    pl.args.zblock = (int)std::min<int64_t>(g.n0, zb);
  }
  pl.name = ac ? (xp ? "stencil3d_xp_acoustic" : "stencil3d_tma_acoustic")
              : (xp ? "stencil3d_xp_diffusion" : "stencil3d_tma_diffusion");
  return cudaSuccess;
}

// One step with u^n in level[cur]; writes u^{n+1} into out (= level[cur ^ 1]).
inline cudaError_t launch_tma_step(const TmaPlan &pl, int cur, float *out, const Coef &c, int *err,
                                   const SparseArgs &sp, cudaStream_t s,
                                   const unsigned char *unit_c = nullptr) {
  TmaArgs a = pl.args;
  a.c = c;
  a.out = out;
  a.err = err;
  a.sp = sp;
  a.unit_c = unit_c;
  pl.fn<<<pl.grid, pl.threads, pl.smem, s>>>(pl.map_u[cur], pl.map_t[cur ^ 1], pl.map_a,
                                              pl.map_c, pl.map_c, pl.map_c, a, BatchArgs{});
  return cudaGetLastError();
}

// The same step with the FWI epilogue (plan.fn_fwi must be set).
inline cudaError_t launch_tma_step_fwi(const TmaPlan &pl, int cur, float *out, const Coef &c,
                                       int *err, const SparseArgs &sp, float *d2, float *img,
                                       const float *img_d2, float img_scale, cudaStream_t s,
                                       const unsigned char *unit_c = nullptr) {
  TmaArgs a = pl.args;
  a.c = c;
  a.out = out;
  a.err = err;
  a.sp = sp;
  a.unit_c = unit_c;
  a.d2 = d2;
  a.img = img;
  a.img_d2 = img_d2;
  a.img_scale = img_scale;
  CUtensorMap me = pl.map_c, mg = pl.map_c;
  if (img) {
    EncodeFn enc = tma_encoder();
    if (!enc || !encode_map(enc, &me, const_cast<float *>(img_d2), pl.args.g, kTmaTX,
                            tma_ty(pl.ny), pl.args.org) ||
        !encode_map(enc, &mg, img, pl.args.g, kTmaTX, tma_ty(pl.ny), pl.args.org))
      return cudaErrorInvalidValue;
  }
  pl.fn_fwi<<<pl.grid, kTmaThreads, pl.smem_fwi, s>>>(pl.map_u[cur], pl.map_t[cur ^ 1], pl.map_a,
                                                      pl.map_c, me, mg, a, BatchArgs{});
  return cudaGetLastError();
}

inline void destroy_tma(TmaPlan &) {}

}  // namespace fdk
