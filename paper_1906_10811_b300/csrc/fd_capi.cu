// fd_capi.cu -- runtime behind the C ABI of include/fd.h.
//
// A context owns: the padded time levels u[2] (rotated by pointer, thesis
// §3.3.2), the acoustic coefficient fields A and C, a dense copy of m for the
// source scaling, the sparse-operator tables, the trace buffer, a device step
// counter, and the cached CUDA graphs of the step loop.  The host time loop of
// an OPS program (one ops_par_loop per step, §3.3.3) becomes one graph replay
// per chunk of steps; nothing crosses the host/device boundary inside a run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/fd.h"
#include "fd_common.cuh"
#include "fd_kernels_plain.cuh"
#include "fd_kernels_tma.cuh"

using namespace fdk;

namespace {

constexpr int kGraphChunk = 64;  // steps per captured graph
// 2-D diffusion grids of at least this many points run the streaming kernel by
// default (measured: 0.88 of the copy bandwidth at 10000² so 2, against 0.36 for the
// plain kernel; the acoustic step, whose coefficients the stream does not stage,
// keeps the plain kernel)
constexpr int64_t kStream2dPoints = 4 << 20;
constexpr int kGraphCacheMax = 12;
thread_local std::string g_create_error;  // fd_last_error(NULL)

// ---------------------------------------------------------------------------
// Weights: closed form of the central second-derivative stencil of order 2r,
//   w_k = 2 (-1)^(k+1) / k² · Π_{i=0}^{k-1} (r-i) / Π_{i=1}^{k} (r+i),
//   w_0 = -2 Σ_{k≥1} w_k,
// evaluated in long double.
// ---------------------------------------------------------------------------
bool lib_weights(int so, double *w) {
  if (so < 2 || so > 2 * kMaxR || (so & 1)) return false;
  const int r = so / 2;
  long double sum = 0.0L;
  for (int k = 1; k <= r; ++k) {
    long double ratio = 1.0L;
    for (int i = 0; i < k; ++i) ratio *= (long double)(r - i) / (long double)(r + i + 1);
    const long double wk = (k % 2 ? 2.0L : -2.0L) / ((long double)k * k) * ratio;
    w[k] = (double)wk;
    sum += wk;
  }
  w[0] = (double)(-2.0L * sum);
  return true;
}

double lib_symbol(int so) {
  double w[kMaxR + 1];
  if (!lib_weights(so, w)) return NAN;
  double s = w[0];
  for (int k = 1; k <= so / 2; ++k) s += 2.0 * (k % 2 ? -w[k] : w[k]);
  return -s;
}

// A sequence of FWI-epilogue steps (fd_run_fwi): step i of nt writes the second
// difference into d2_base + s(i)·stride and/or accumulates the imaging condition
// into img reading img_d2_base + s(i)·stride, s(i) = i or nt-1-i (reverse).
struct FwiSeq {
  float *d2_base = nullptr;
  const float *img_d2_base = nullptr;
  float *img = nullptr;
  int64_t stride = 0;
  int64_t nt = 0, i0 = 0;  // steps in the sequence; index of the chunk's first step
  int reverse = 0;
  float scale = 0.f;
  bool operator==(const FwiSeq &o) const {
    return d2_base == o.d2_base && img_d2_base == o.img_d2_base && img == o.img &&
           stride == o.stride && nt == o.nt && i0 == o.i0 && reverse == o.reverse &&
           std::memcmp(&scale, &o.scale, sizeof scale) == 0;
  }
};

struct GraphEntry {
  int parity;
  int len;
  int64_t kernels;  // kernel nodes in the graph
  cudaGraphExec_t exec;
  bool fwi;         // captured with an FWI-epilogue sequence (key below)
  FwiSeq seq;
};

using StencilFn = void (*)(const float *, float *, const float *, const float *, Geom, Coef);
using StencilFnStream = void (*)(const float *, float *, const float *, const float *, Geom, Coef,
                                 int, int);
using StencilFnStream2 = void (*)(const float *, float *, Geom, Coef, int, int);
using StencilFn2D = void (*)(const MemberDesc *, int, const int64_t *, int);

}  // namespace

struct fd_ctx {
  // problem
  int ndim = 0;
  int64_t shape[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  int so = 0;
  double dt = 0;
  fd_equation eq = FD_DIFFUSION;
  fd_options opt{};
  Geom g{};
  Coef coef{};
  int nc = 0;  // 2^ndim corners
  // device
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *u[2] = {nullptr, nullptr};
  int cur = 0;  // u[cur] = u^n, u[cur ^ 1] = u^{n-1}
  float *A = nullptr, *C = nullptr, *m_dense = nullptr, *stage = nullptr;
  int64_t *d_step = nullptr;
  unsigned *d_stats = nullptr;
  int *d_err = nullptr;
  // kernel selection
  StencilFn plain_fn = nullptr;
  StencilFnStream stream2d_fn = nullptr;  // 2-D grids: rows staged and streamed along y
  // 2-D diffusion, radius 1-2, zero halo: two steps a launch (u^{n+2} from u^n)
  StencilFnStream2 stream2d2_fn = nullptr;
  int s2_nseg = 0, s2_seglen = 0;         // its row segments per strip and their length
  int s2_p = 1;                           // its pairs a lane, adjacent (strips 64·s2_p wide)
  int s2t_nseg = 0, s2t_seglen = 0;       // the same for the two-step stream (strips s2t_w(P) wide)
  int s2t_p = 1;                          // its pairs a lane
  TmaPlan tma{};
  bool use_tma = false;
  bool iso = false;          // equal spacing on all axes (pipelined kernel variant)
  double tune_us = 0.0;      // stencil µs of the current tile configuration, if measured
  // FWI epilogue of the step fd_step_fwi launches (see launch_stencil)
  bool fwi_on = false;
  float *fwi_d2 = nullptr, *fwi_img = nullptr;
  const float *fwi_img_d2 = nullptr;
  bool fwi_seq_on = false;  // fd_run_fwi: per-step pointers from fwi_seq
  FwiSeq fwi_seq;
  double *fwi_partial = nullptr;  // fd_residual's per-block sums
  float fwi_scale = 0.f;
  const char *kernel_name = "none";
  // sources
  int nsrc = 0, nt_wav = 0;
  float *wav = nullptr, *src_scale = nullptr;
  int64_t *src_off = nullptr, *src_dense = nullptr;
  double *src_w = nullptr;
  bool src_dirty = false;
  // receivers
  int nrec = 0;
  int64_t *rec_off = nullptr;
  float *rec_w = nullptr, *rec = nullptr;
  int64_t rec_cap = 0;   // rows
  int64_t rec_rows = 0;  // rows recorded (valid)
  // pipelined path: injection fused into the stencil epilogue, receivers
  // sampled by a side-stream kernel that overlaps the next step's stencil
  std::vector<int64_t> h_src_dense;  // source corner nodes (dense index)
  int4 *sp_entries = nullptr;
  int *sp_first = nullptr;
  size_t sp_entries_n = 0, sp_first_n = 0;  // their lengths
  bool sp_dirty = true;
  // tile-planes of the pipelined kernel where C = 1 (no damping): their C tile is skipped
  unsigned char *unit_c = nullptr;
  size_t unit_c_cap = 0;
  bool unit_c_dirty = true;
  bool skip_c = false;  // fd_tile_config.skip_c
  bool fused = false;                // this run uses the fused/overlapped sparse path
  cudaStream_t side = nullptr;
  // host mode: model uploads run on their own stream, so that they overlap steps
  // still in flight on the context stream; ev_model_free is recorded after every
  // queued reader of m_dense and stage, ev_copied after an upload
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_model_free = nullptr, ev_copied = nullptr;
  cudaEvent_t ev_step[2] = {nullptr, nullptr}, ev_rec[2] = {nullptr, nullptr};
  // z-slab sub-domain (fd_set_subdomain): this context holds global z nodes
  // [z_origin, z_origin + n0) of a grid of z_global nodes (0: the whole grid)
  int64_t z_origin = 0, z_global = 0;
  cudaEvent_t ev_halo = nullptr;  // orders halo copies with a neighbour on another stream
  // state
  bool model_set = false;
  int64_t step = 0;
  bool failed = false;
  std::string err;
  std::vector<GraphEntry> graphs;
  // profiling
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  std::vector<int> ev_launches;  // stencil launches between event pair i (ev[2i], ev[2i+1])
  int64_t launches = 0;  // kernels this context has launched (graph nodes included)
};

namespace {

fd_status fail(fd_ctx *c, fd_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (st == FD_ECUDA) c->failed = true;
  } else {
    g_create_error = buf;
  }
  return st;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(c, e_ == cudaErrorMemoryAllocation ? FD_ENOMEM : FD_ECUDA,           \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                     \
  } while (0)

#define CHECK_LAUNCH()   \
  do {                   \
    CU(cudaGetLastError()); \
    ++c->launches;       \
  } while (0)

fd_status check_usable(fd_ctx *c) {
  if (!c) return FD_EINVAL;
  if (c->failed) return FD_ECUDA;
  CU(cudaSetDevice(c->device));
  return FD_OK;
}

// Context memory comes from the device's stream-ordered pool on the context
// stream: admitting or retiring a shot does not synchronise the device.
template <typename T>
fd_status dalloc(fd_ctx *c, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocAsync((void **)p, count * sizeof(T), c->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? FD_ENOMEM : FD_ECUDA,
                "cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
  }
  return FD_OK;
}

template <typename T>
void dfree(fd_ctx *c, T *&p) {
  if (p) cudaFreeAsync(p, c->stream);
  p = nullptr;
}

void drop_graphs(fd_ctx *c) {
  for (auto &gph : c->graphs) cudaGraphExecDestroy(gph.exec);
  c->graphs.clear();
}

// Copy n elements of user data (host or device per options) to a device buffer.
template <typename T>
fd_status to_device(fd_ctx *c, T *dst, const T *src, size_t n) {
  if (n == 0) return FD_OK;
  CU(cudaMemcpyAsync(dst, src, n * sizeof(T),
                     c->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream));
  return FD_OK;
}

// User coordinates (host or device) -> host vector.
fd_status coords_to_host(fd_ctx *c, const float *src, size_t n, std::vector<float> &out) {
  out.resize(n);
  if (n == 0) return FD_OK;
  if (c->opt.device_ptrs) {
    CU(cudaMemcpyAsync(out.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(out.data(), src, n * sizeof(float));
  }
  return FD_OK;
}

int blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 32));
}

// Host mode: the work queued so far that reads m_dense or stage ends here.
fd_status model_readers_queued(fd_ctx *c) {
  if (c->ev_model_free) CU(cudaEventRecord(c->ev_model_free, c->stream));
  return FD_OK;
}

// Scatter a dense interior array (host or device) into a padded field: one
// upload, scattered into `padded` and, if given, into `padded2` as well.
fd_status load_field(fd_ctx *c, float *padded, const float *user, float *padded2 = nullptr) {
  const size_t n = (size_t)c->g.n0 * c->g.n1 * c->g.n2;
  const float *src = user;
  if (!c->opt.device_ptrs) {
    CU(cudaMemcpyAsync(c->stage, user, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    src = c->stage;
  }
  k_scatter<<<blocks_for(n, 256), 256, 0, c->stream>>>(src, padded, c->g);
  CHECK_LAUNCH();
  if (padded2) {
    k_scatter<<<blocks_for(n, 256), 256, 0, c->stream>>>(src, padded2, c->g);
    CHECK_LAUNCH();
  }
  return model_readers_queued(c);
}

fd_status store_field(fd_ctx *c, const float *padded, float *user) {
  const size_t n = (size_t)c->g.n0 * c->g.n1 * c->g.n2;
  float *dst = c->opt.device_ptrs ? user : c->stage;
  k_gather<<<blocks_for(n, 256), 256, 0, c->stream>>>(padded, dst, c->g);
  CHECK_LAUNCH();
  if (!c->opt.device_ptrs)
    CU(cudaMemcpyAsync(user, c->stage, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  return model_readers_queued(c);
}

// Multilinear corners of one point (the rule documented in fd.h).
// In a z-slab sub-domain the point is placed on the global grid and a corner
// whose node lies in another slab gets dense index -1, padded offset 0 and
// weight 0 (its owner adds it).
bool corners(const fd_ctx *c, const float *pt, int64_t *pad_off, int64_t *dense_idx, double *w) {
  int64_t i[3] = {0, 0, 0};
  double f[3] = {0, 0, 0};
  for (int d = 0; d < c->ndim; ++d) {
    const int64_t n = (d == 0 && c->z_global > 0) ? c->z_global : c->shape[d];
    if (n < 2) return false;
    double x = (double)pt[d] / c->h[d];
    const double last = (double)(n - 1), tol = 1e-9 * last;
    if (!(x >= -tol && x <= last + tol)) return false;
    x = std::min(std::max(x, 0.0), last);
    i[d] = (int64_t)std::floor(x);
    f[d] = x - (double)i[d];
    if (i[d] == n - 1) {
      i[d] = n - 2;
      f[d] = 1.0;
    }
  }
  for (int b = 0; b < c->nc; ++b) {
    int64_t node[3] = {0, 0, 0};
    double wt = 1.0;
    for (int d = 0; d < c->ndim; ++d) {
      const int bit = (b >> (c->ndim - 1 - d)) & 1;
      node[d] = i[d] + bit;
      wt *= bit ? f[d] : 1.0 - f[d];
    }
    int z, y, x;
    if (c->ndim == 3) {
      z = (int)(node[0] - c->z_origin); y = (int)node[1]; x = (int)node[2];
    } else {
      z = 0; y = (int)node[0]; x = (int)node[1];
    }
    if (c->z_global > 0 && (z < 0 || z >= c->g.n0)) {  // another slab's node
      pad_off[b] = 0;
      dense_idx[b] = -1;
      w[b] = 0.0;
      continue;
    }
    pad_off[b] = gidx(c->g, z, y, x);
    dense_idx[b] = ((int64_t)z * c->g.n1 + y) * c->g.n2 + x;
    w[b] = wt;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Launching one step.
// ---------------------------------------------------------------------------
fd_status launch_stencil(fd_ctx *c, const float *ucur, float *unext, int j) {
  if (c->fwi_seq_on) {  // step j of the chunk: pointers of sequence step i0 + j
    const FwiSeq &q = c->fwi_seq;
    const int64_t i = q.i0 + j, s = q.reverse ? q.nt - 1 - i : i;
    c->fwi_d2 = q.d2_base ? q.d2_base + s * q.stride : nullptr;
    c->fwi_img_d2 = q.img_d2_base ? q.img_d2_base + s * q.stride : nullptr;
    c->fwi_img = q.img;
    c->fwi_scale = q.scale;
  }
  if (c->use_tma) {
    SparseArgs sp{};
    if (c->fused && c->nsrc > 0) {
      sp.entries = c->sp_entries;
      sp.first = c->sp_first;
      sp.src_scale = c->src_scale;
      sp.wav = c->wav;
      sp.step = c->d_step;
      sp.j = j;
      sp.nsrc = c->nsrc;
      sp.nc = c->nc;
    }
    const int cur = ucur == c->u[0] ? 0 : 1;
    const unsigned char *uc = c->skip_c ? c->unit_c : nullptr;
    cudaError_t e =
        c->fwi_on ? launch_tma_step_fwi(c->tma, cur, unext, c->coef, c->d_err, sp, c->fwi_d2,
                                        c->fwi_img, c->fwi_img_d2, c->fwi_scale, c->stream, uc)
                  : launch_tma_step(c->tma, cur, unext, c->coef, c->d_err, sp, c->stream, uc);
    if (e != cudaSuccess) return fail(c, FD_ECUDA, "TMA stencil launch: %s", cudaGetErrorString(e));
    ++c->launches;
    return FD_OK;
  }
  dim3 block(32, 8);
  if (c->stream2d_fn) {
    const int w = kS2W * c->s2_p;
    const int64_t items = (int64_t)((c->g.n2 + w - 1) / w) * c->s2_nseg;
    const int nw = s2_warps(c->g.R);
    c->stream2d_fn<<<(unsigned)((items + nw - 1) / nw), nw * 32, s2_smem(c->g.R, c->s2_p),
                     c->stream>>>(
        ucur, unext, c->A, c->C, c->g, c->coef, c->s2_nseg, c->s2_seglen);
    CHECK_LAUNCH();
    return FD_OK;
  }
  dim3 grid((c->g.n2 + 31) / 32, (c->g.n1 + 7) / 8, c->g.n0);
  c->plain_fn<<<grid, block, 0, c->stream>>>(ucur, unext, c->A, c->C, c->g, c->coef);
  CHECK_LAUNCH();
  return FD_OK;
}

// Two steps in one launch (the 2-D diffusion stream): u^{n+2} from ucur into unext.
fd_status launch_stencil2(fd_ctx *c, const float *ucur, float *unext) {
  const int w = s2t_w(c->s2t_p);
  const int64_t items = (int64_t)((c->g.n2 + w - 1) / w) * c->s2t_nseg;
  const int nw = s2_warps(c->g.R);
  c->stream2d2_fn<<<(unsigned)((items + nw - 1) / nw), nw * 32, s2t_smem(c->g.R, c->s2t_p),
                    c->stream>>>(
      ucur, unext, c->g, c->coef, c->s2t_nseg, c->s2t_seglen);
  CHECK_LAUNCH();
  ++c->launches;
  return FD_OK;
}

// Level flips of a chunk of len steps: one per launch (two-step launches cover pairs).
int chunk_flips(const fd_ctx *c, int len) { return c->stream2d2_fn ? len / 2 + (len & 1) : len; }

// Source injection of step j into unext (kernels without the fused epilogue).
fd_status launch_inject(fd_ctx *c, float *unext, int j) {
  const int n = c->nsrc * c->nc;
  if (c->nc == 8)
    k_inject<8><<<(n + 255) / 256, 256, 0, c->stream>>>(unext, c->d_step, j, c->nsrc, c->src_off,
                                                         c->src_scale, c->wav);
  else
    k_inject<4><<<(n + 255) / 256, 256, 0, c->stream>>>(unext, c->d_step, j, c->nsrc, c->src_off,
                                                         c->src_scale, c->wav);
  CHECK_LAUNCH();
  return FD_OK;
}

// Record row 0 = interp(u^0) (needs *d_step = 0).
fd_status launch_interp_row0(fd_ctx *c) {
  const int n = c->nrec * c->nc;
  if (c->nc == 8)
    k_interp<8><<<(n + 255) / 256, 256, 0, c->stream>>>(c->u[c->cur], c->d_step, -1, c->nrec,
                                                         c->rec_off, c->rec_w, c->rec);
  else
    k_interp<4><<<(n + 255) / 256, 256, 0, c->stream>>>(c->u[c->cur], c->d_step, -1, c->nrec,
                                                         c->rec_off, c->rec_w, c->rec);
  CHECK_LAUNCH();
  return FD_OK;
}

// Steps j = 0..len-1 of a chunk starting with u^n in u[parity]; ends by
// advancing the device step counter by len.
// Receiver samples of step j (row n+1) from unext on the side stream; the
// stencil that next overwrites unext (step j+2) waits for it.
fd_status launch_receivers_side(fd_ctx *c, float *unext, int j) {
  CU(cudaEventRecord(c->ev_step[j & 1], c->stream));
  CU(cudaStreamWaitEvent(c->side, c->ev_step[j & 1], 0));
  const int n = c->nrec * c->nc;
  if (c->nc == 8)
    k_interp<8><<<(n + 255) / 256, 256, 0, c->side>>>(unext, c->d_step, j, c->nrec, c->rec_off,
                                                       c->rec_w, c->rec);
  else
    k_interp<4><<<(n + 255) / 256, 256, 0, c->side>>>(unext, c->d_step, j, c->nrec, c->rec_off,
                                                       c->rec_w, c->rec);
  CHECK_LAUNCH();
  CU(cudaEventRecord(c->ev_rec[j & 1], c->side));
  return FD_OK;
}

// Profile mode: an event pair around a stretch of `launches` stencil launches.
fd_status profile_mark(fd_ctx *c, bool end, int launches) {
  if (!end && c->ev_used + 2 > c->ev.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      CU(cudaEventCreate(&e));
      c->ev.push_back(e);
    }
  }
  CU(cudaEventRecord(c->ev[c->ev_used + (end ? 1 : 0)], c->stream));
  if (end) {
    c->ev_launches.resize(c->ev_used / 2 + 1);
    c->ev_launches[c->ev_used / 2] = launches;
    c->ev_used += 2;
  }
  return FD_OK;
}

fd_status enqueue_chunk(fd_ctx *c, int parity, int len, bool timed) {
  const bool overlap = c->fused && c->nrec > 0;
  int b = parity;  // level holding u^n of step j
  for (int j = 0; j < len; ++j, b ^= 1) {
    float *ucur = c->u[b], *unext = c->u[b ^ 1];
    if (c->stream2d2_fn && j + 1 < len) {
      // steps j and j+1 in one launch (2-D diffusion: no odd halo, sources or receivers)
      fd_status st = timed ? profile_mark(c, false, 0) : FD_OK;
      if (!st) st = launch_stencil2(c, ucur, unext);
      if (!st && timed) st = profile_mark(c, true, 2);
      if (st) return st;
      ++j;
      continue;
    }
    if (overlap && j >= 2) CU(cudaStreamWaitEvent(c->stream, c->ev_rec[j & 1], 0));
    if (c->opt.boundary == FD_BOUNDARY_ODD) {
      // halo of u^n = odd mirror of the interior about the boundary nodes
      const int64_t cells = 2LL * c->g.R *
                            ((c->g.R0 ? (int64_t)c->g.n1 * c->g.n2 : 0) +
                             (int64_t)c->g.n0 * c->g.n2 + (int64_t)c->g.n0 * c->g.n1);
      k_odd_halo<<<(unsigned)std::min<int64_t>((cells + 255) / 256, 4096), 256, 0, c->stream>>>(
          ucur, c->g);
      CHECK_LAUNCH();
    }
    fd_status st = timed ? profile_mark(c, false, 0) : FD_OK;
    if (st) return st;
    st = launch_stencil(c, ucur, unext, j);
    if (st) return st;
    st = timed ? profile_mark(c, true, 1) : FD_OK;
    if (st) return st;
    if (c->fused && !c->use_tma && c->nsrc)
      st = launch_inject(c, unext, j);  // the stencil has no injection epilogue here
    if (!st && overlap) st = launch_receivers_side(c, unext, j);
    if (st) return st;
  }
  if (overlap) {  // join the side stream before the step counter moves
    CU(cudaStreamWaitEvent(c->stream, c->ev_rec[(len - 1) & 1], 0));
    if (len >= 2) CU(cudaStreamWaitEvent(c->stream, c->ev_rec[len & 1], 0));
  }
  k_advance_step<<<1, 1, 0, c->stream>>>(c->d_step, len);
  CHECK_LAUNCH();
  return FD_OK;
}

fd_status get_graph(fd_ctx *c, int parity, int len, cudaGraphExec_t *out, int64_t *kernels) {
  for (auto &gph : c->graphs)
    if (gph.parity == parity && gph.len == len && gph.fwi == c->fwi_seq_on &&
        (!gph.fwi || gph.seq == c->fwi_seq)) {
      *out = gph.exec;
      *kernels = gph.kernels;
      return FD_OK;
    }
  if ((int)c->graphs.size() >= kGraphCacheMax) {
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  cudaGraph_t graph;
  CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  const int64_t before = c->launches;
  fd_status st = enqueue_chunk(c, parity, len, false);
  const int64_t captured = c->launches - before;
  c->launches = before;  // counted when the graph is replayed
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (st) {
    if (e == cudaSuccess) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(c, FD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(c, FD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graphs.push_back({parity, len, captured, exec, c->fwi_seq_on, c->fwi_seq});
  *out = exec;
  *kernels = captured;
  return FD_OK;
}

// Make the trace buffer hold at least `rows` rows (keeps recorded rows).
fd_status ensure_rec_capacity(fd_ctx *c, int64_t rows) {
  if (c->nrec == 0 || rows <= c->rec_cap) return FD_OK;
  int64_t cap = std::max<int64_t>(rows, std::max<int64_t>(2 * c->rec_cap, 1024));
  float *nb = nullptr;
  fd_status st = dalloc(c, &nb, (size_t)cap * c->nrec);
  if (st) return st;
  cudaError_t e = cudaMemsetAsync(nb, 0, (size_t)cap * c->nrec * sizeof(float), c->stream);
  if (e == cudaSuccess && c->rec && c->rec_rows > 0)
    e = cudaMemcpyAsync(nb, c->rec, (size_t)c->rec_rows * c->nrec * sizeof(float),
                        cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(nb, c->stream);
    return fail(c, FD_ECUDA, "trace buffer growth: %s", cudaGetErrorString(e));
  }
  CU(cudaStreamSynchronize(c->stream));
  dfree(c, c->rec);
  c->rec = nb;
  c->rec_cap = cap;
  drop_graphs(c);
  return FD_OK;
}

fd_status prepare_sources(fd_ctx *c) {
  if (!c->src_dirty || c->nsrc == 0) return FD_OK;
  const int n = c->nsrc * c->nc;
  k_source_scales<<<(n + 255) / 256, 256, 0, c->stream>>>(c->src_dense, c->src_w, c->m_dense,
                                                           c->src_scale, n, c->dt);
  CHECK_LAUNCH();
  c->src_dirty = false;
  return model_readers_queued(c);
}

// Pipelined path: the source corners as entries keyed by (tile, plane) of the
// pipelined kernel; receivers need only the side stream and its events.
// Other kernels (2-D, plain): receivers on the side stream as well, sources by
// k_inject after the stencil (no entry table).
fd_status prepare_fused(fd_ctx *c) {
  c->fused = false;
  if (c->eq != FD_ACOUSTIC || (c->nsrc == 0 && c->nrec == 0)) return FD_OK;
  if (!c->side) {
    CU(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CU(cudaEventCreateWithFlags(&c->ev_step[i], cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&c->ev_rec[i], cudaEventDisableTiming));
    }
  }
  if (c->sp_dirty && c->use_tma) {
    const int ty = tma_ty(c->tma.ny), tiles_x = c->tma.args.tiles_x;
    struct E { int64_t key; int idx, x, y, z; };
    std::vector<E> es;
    for (size_t i = 0; i < c->h_src_dense.size(); ++i) {
      const int64_t d = c->h_src_dense[i];
      if (d < 0) continue;  // a corner another z-slab owns
      const int x = (int)(d % c->g.n2);
      const int y = (int)((d / c->g.n2) % c->g.n1);
      const int z = (int)(d / ((int64_t)c->g.n1 * c->g.n2));
      const int tile = (y / ty) * tiles_x + x / c->tma.tx;
      es.push_back({(int64_t)tile * c->g.n0 + z, (int)i, x, y, z});
    }
    std::sort(es.begin(), es.end(), [](const E &a, const E &b) {
      return a.key != b.key ? a.key < b.key : a.idx < b.idx;
    });
    const int64_t nkeys = (int64_t)c->g.n0 * c->tma.args.ntiles;
    std::vector<int> first(nkeys + 1, 0);
    for (const E &e : es) ++first[e.key + 1];
    for (int64_t k = 0; k < nkeys; ++k) first[k + 1] += first[k];
    std::vector<int4> ent(es.size());
    for (size_t i = 0; i < es.size(); ++i) ent[i] = make_int4(es[i].x, es[i].y, es[i].z, es[i].idx);
    CU(cudaStreamSynchronize(c->stream));
    const size_t nfirst = es.empty() ? 0 : first.size();
    if (ent.size() != c->sp_entries_n || nfirst != c->sp_first_n) {
      dfree(c, c->sp_entries);
      dfree(c, c->sp_first);
      c->sp_entries_n = c->sp_first_n = 0;
      drop_graphs(c);
      if (!es.empty()) {
        fd_status st = dalloc(c, &c->sp_entries, ent.size());
        if (!st) st = dalloc(c, &c->sp_first, first.size());
        if (st) return st;
        c->sp_entries_n = ent.size();
        c->sp_first_n = first.size();
      }
    }
    if (!es.empty()) {
      CU(cudaMemcpyAsync(c->sp_entries, ent.data(), ent.size() * sizeof(int4),
                         cudaMemcpyHostToDevice, c->stream));
      CU(cudaMemcpyAsync(c->sp_first, first.data(), first.size() * sizeof(int),
                         cudaMemcpyHostToDevice, c->stream));
      CU(cudaStreamSynchronize(c->stream));
    }
    c->sp_dirty = false;
  }
  c->fused = true;
  return FD_OK;
}

// Flags of the tile-planes where C = 1 for the current plan (acoustic pipelined
// kernel); recomputed after fd_set_model or a new tile configuration.
fd_status prepare_unit_c(fd_ctx *c) {
  if (!c->use_tma || !c->skip_c || !c->unit_c_dirty) return FD_OK;
  const size_t n = (size_t)c->tma.args.ntiles * c->g.n0;
  if (n > c->unit_c_cap) {
    drop_graphs(c);  // the captured launches hold the flags pointer
    dfree(c, c->unit_c);
    c->unit_c_cap = 0;
    fd_status st = dalloc(c, &c->unit_c, n);
    if (st) return st;
    c->unit_c_cap = n;
  }
  k_unit_c<<<(unsigned)n, 128, 0, c->stream>>>(c->C, c->g, c->tma.args.tiles_x, c->tma.tx,
                                               tma_ty(c->tma.ny), c->unit_c);
  CHECK_LAUNCH();
  c->unit_c_dirty = false;
  return FD_OK;
}

void select_kernel(fd_ctx *c) {
  const int R = c->so / 2;
  const bool three = c->ndim == 3;
  const bool ac = c->eq == FD_ACOUSTIC;
  const bool iso2 = !three && c->coef.iso2;
#define PICK(RR)                                                                       \
  case RR:                                                                             \
    c->plain_fn = three ? (ac ? k_stencil_plain<RR, kAcoustic, true>                   \
                              : k_stencil_plain<RR, kDiffusion, true>)                 \
                  : iso2 ? (ac ? k_stencil_plain<RR, kAcoustic, false, true>           \
                               : k_stencil_plain<RR, kDiffusion, false, true>)         \
                         : (ac ? k_stencil_plain<RR, kAcoustic, false>                 \
                               : k_stencil_plain<RR, kDiffusion, false>);              \
    break;
  switch (R) {
    PICK(1) PICK(2) PICK(3) PICK(4) PICK(5) PICK(6) PICK(7) PICK(8)
  }
#undef PICK
  c->kernel_name = three ? "stencil3d_plain" : "stencil2d_plain";
  c->stream2d_fn = nullptr;
  c->stream2d2_fn = nullptr;
  if (!three) {
    // rows staged and streamed along y: on request (FD_KERNEL_TMA), and by default for
    // diffusion on grids too large for L2, where one thread per point keeps too few
    // bytes in flight to fill HBM
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 148;
    }
    const int64_t pts = (int64_t)c->g.n1 * c->g.n2;
    const bool want = c->opt.kernel == FD_KERNEL_TMA ||
                      (c->opt.kernel == FD_KERNEL_AUTO && !ac && pts >= kStream2dPoints);
    if (want) {
#define PICK2(RR)                                                                      \
  case RR:                                                                             \
    c->stream2d_fn = iso2 ? (ac ? k_stencil2d_stream<RR, kAcoustic, true>              \
                                : k_stencil2d_stream<RR, kDiffusion, true>)            \
                          : (ac ? k_stencil2d_stream<RR, kAcoustic>                    \
                                : k_stencil2d_stream<RR, kDiffusion>);                 \
    cudaFuncSetAttribute((const void *)c->stream2d_fn,                                 \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, s2_smem(RR));    \
    break;
      switch (R) {
        PICK2(1) PICK2(2) PICK2(3) PICK2(4) PICK2(5) PICK2(6) PICK2(7) PICK2(8)
      }
#undef PICK2
      // about 64 warp streams per SM in all (measured ahead of sizing the grid to one
      // wave of the occupancy: 0.88 against 0.81 of the copy bandwidth at 10000² so 2),
      // segments of at least max(32, 4R) rows
      const int most = std::max(1, c->g.n1 / std::max(32, 4 * R));
      // diffusion at radius 2-7: four adjacent points a lane (128-column strips, 16-byte
      // shared-memory reads and stores, the per-row work shared by twice the points)
      // where the grid has the strips and segments for those streams (10000²: so 8
      // 172.7 -> 148.6 µs, so 12 202.1 -> 163.1, so 14 212.3 -> 203.3; at radius 1 and 8
      // one pair a lane was as fast or faster)
      c->s2_p = 1;
      if (!ac && R >= 2 && R <= 7 &&
          (int64_t)((c->g.n2 + 2 * kS2W - 1) / (2 * kS2W)) * most >= 64 * sms) {
        StencilFnStream f2 = nullptr;
#define PICK2P(RR)                                                                     \
  case RR:                                                                             \
    f2 = iso2 ? k_stencil2d_stream<RR, kDiffusion, true, 2>                            \
              : k_stencil2d_stream<RR, kDiffusion, false, 2>;                          \
    break;
        switch (R) {
          PICK2P(2) PICK2P(3) PICK2P(4) PICK2P(5) PICK2P(6) PICK2P(7)
        }
#undef PICK2P
        if (f2 && cudaFuncSetAttribute((const void *)f2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       s2_smem(R, 2)) == cudaSuccess) {
          c->stream2d_fn = f2;
          c->s2_p = 2;
        } else {
          cudaGetLastError();
        }
      }
      const int strips = (c->g.n2 + kS2W * c->s2_p - 1) / (kS2W * c->s2_p);
      const int nseg = std::max(1, std::min((64 * sms + strips - 1) / strips, most));
      c->s2_seglen = (c->g.n1 + nseg - 1) / nseg;
      c->s2_nseg = (c->g.n1 + c->s2_seglen - 1) / c->s2_seglen;
      c->kernel_name = "stencil2d_stream";
      // diffusion at radius 1-2 with the zero halo: pairs of steps in one pass (the
      // step moves 8 bytes a point and has compute to spare; two steps move 8 in all)
      if (!ac && R <= 2 && c->opt.boundary != FD_BOUNDARY_ODD) {
        // two pairs a lane (124-column strips, half the per-row work a point) where the
        // grid has the strips and segments to fill a wave with them; one pair otherwise
        auto pick = [&](int P) -> StencilFnStream2 {
          if (R == 1)
            return P == 2 ? (iso2 ? k_stencil2d_stream2<1, true, 2> : k_stencil2d_stream2<1, false, 2>)
                          : (iso2 ? k_stencil2d_stream2<1, true, 1> : k_stencil2d_stream2<1, false, 1>);
          return P == 2 ? (iso2 ? k_stencil2d_stream2<2, true, 2> : k_stencil2d_stream2<2, false, 2>)
                        : (iso2 ? k_stencil2d_stream2<2, true, 1> : k_stencil2d_stream2<2, false, 1>);
        };
        // streams a wave holds (segments of at least 32 rows) for P pairs a lane
        auto wave = [&](int P, StencilFnStream2 fn, int *streams) {
          int per_sm = 0;
          cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               s2t_smem(R, P));
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn,
                                                            s2_warps(R) * 32, s2t_smem(R, P)) !=
                  cudaSuccess ||
              per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
          }
          *streams = per_sm * s2_warps(R) * sms;
        };
        const int most2 = std::max(1, c->g.n1 / 32);
        int streams2 = 0;
        wave(2, pick(2), &streams2);
        const int64_t items2 = (int64_t)((c->g.n2 + s2t_w(2) - 1) / s2t_w(2)) * most2;
        c->s2t_p = items2 >= streams2 ? 2 : 1;
        c->stream2d2_fn = pick(c->s2t_p);
        int streams = streams2;
        if (c->s2t_p == 1) wave(1, c->stream2d2_fn, &streams);
        // segments for one wave of the kernel's own occupancy, at least 32 rows
        const int strips2 = (c->g.n2 + s2t_w(c->s2t_p) - 1) / s2t_w(c->s2t_p);
        const int nseg2 = (int)std::max<int64_t>(1, std::min<int64_t>(streams / strips2, most2));
        c->s2t_seglen = (c->g.n1 + nseg2 - 1) / nseg2;
        c->s2t_nseg = (c->g.n1 + c->s2t_seglen - 1) / c->s2t_seglen;
        c->kernel_name = "stencil2d_stream2";
      }
    }
  }
}

// Tensor-map origin of the context's fields (see map_origin).
MapOrigin ctx_origin(const fd_ctx *c) {
  return map_origin(c->g, c->opt.boundary == FD_BOUNDARY_ODD, c->z_global > 0);
}

// Rebuild the pipelined kernel's plan for another tile configuration; on
// failure the current plan stays.  Source tables are keyed by tile and the
// captured graphs hold the old plan, so both are redone.
fd_status replan(fd_ctx *c, int ny, int per_sm, int zblock, int aligned, int skip_c = 0,
                 int tx = kTmaTX) {
  TmaPlan p{};
  const char *why = nullptr;
  cudaError_t e = plan_tma(p, c->g, c->eq == FD_ACOUSTIC ? kAcoustic : kDiffusion, c->iso, c->u,
                           c->A, c->C, ny, per_sm, zblock, aligned, &why, tx, ctx_origin(c));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorInvalidValue ? FD_EINVAL : FD_EUNSUPPORTED,
                "tile configuration: %s", why ? why : cudaGetErrorString(e));
  }
  CU(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  c->tma = p;
  c->kernel_name = c->tma.name;  // the variant fd_run now launches (tile width)
  c->skip_c = skip_c && c->eq == FD_ACOUSTIC && c->g.R <= 4;
  c->sp_dirty = true;
  c->unit_c_dirty = true;
  c->tune_us = 0.0;
  return FD_OK;
}

void tile_of(const fd_ctx *c, fd_tile_config *cfg) {
  cfg->tile_x = c->tma.tx;
  cfg->tile_y = tma_ty(c->tma.ny);
  cfg->zblock = c->tma.args.zblock;
  cfg->ctas_per_sm = c->tma.per_sm;
  cfg->aligned = c->tma.args.aligned;
  cfg->skip_c = c->skip_c ? 1 : 0;
  cfg->us_per_step = c->tune_us;
}

// Work split a new context starts with (fd_tile_config.aligned): whole segments
// for the acoustic step (measured best or within 3% of it at 128³-512³, so 4-16),
// equal tile-plane ranges for diffusion (6% ahead at 512³ so 8).
inline int default_aligned(fd_equation eq) { return eq == FD_ACOUSTIC ? 1 : 0; }

// Autotuner choices for the process, per device, grid, order and equation.
struct TuneKey {
  int device, so, eq, iso, fwi;
  int64_t n0, n1, n2;
  bool operator<(const TuneKey &o) const {
    return std::tie(device, so, eq, iso, fwi, n0, n1, n2) <
           std::tie(o.device, o.so, o.eq, o.iso, o.fwi, o.n0, o.n1, o.n2);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, fd_tile_config> g_tune_cache;

TuneKey tune_key(const fd_ctx *c, bool fwi) {
  return TuneKey{c->device, c->so, (int)c->eq, c->iso ? 1 : 0, fwi ? 1 : 0,
                 c->g.n0, c->g.n1, c->g.n2};
}

fd_status autotune_impl(fd_ctx *c, int reps, fd_tile_config *best, fd_tile_config *tried,
                        int max_tried, int *ntried, bool fwi = false);

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void fd_options_default(fd_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->nu = 0.5;
  o->use_graphs = 1;
  o->kernel = FD_KERNEL_AUTO;
  o->dirichlet_interior = 1;
}

const char *fd_version(void) { return "fd_b300 0.1 (sm_103a)"; }

fd_status fd_selftest_bounded_wait(double budget_ms, int *expired, double *waited_ms) {
  fd_ctx *c = nullptr;
  if (!expired || !(budget_ms > 0.0) || budget_ms > 10000.0)
    return fail(nullptr, FD_EINVAL, "budget_ms must be in (0, 10000]");
  int dev = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  int *d_out = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void **)&d_out, 2 * sizeof(int));
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 32>>>((long long)(budget_ms * (double)khz), d_out);
    e = cudaGetLastError();
  }
  int out[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof out, cudaMemcpyDeviceToHost);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) return fail(c, FD_ECUDA, "self-test: %s", cudaGetErrorString(e));
  *expired = out[0];
  if (waited_ms) *waited_ms = (double)out[1] * 1024.0 / (double)khz;
  return FD_OK;
}

fd_status fd_weights(int space_order, double *w) {
  if (!w) return FD_EINVAL;
  return lib_weights(space_order, w) ? FD_OK : FD_EINVAL;
}

double fd_stability_symbol(int space_order) { return lib_symbol(space_order); }

fd_status fd_create(fd_ctx **out, int ndim, const int64_t *shape, const double *spacing,
                    int space_order, double dt, fd_equation eq, const fd_options *opt) {
  fd_ctx *c = nullptr;
  if (!out) return fail(nullptr, FD_EINVAL, "out is NULL");
  *out = nullptr;
  g_create_error.clear();
  if (ndim != 2 && ndim != 3) return fail(nullptr, FD_EINVAL, "ndim must be 2 or 3 (got %d)", ndim);
  if (!shape || !spacing) return fail(nullptr, FD_EINVAL, "shape/spacing is NULL");
  if (eq != FD_DIFFUSION && eq != FD_ACOUSTIC)
    return fail(nullptr, FD_EINVAL, "unknown equation %d", (int)eq);
  if (space_order < 2 || space_order > 2 * kMaxR || (space_order & 1))
    return fail(nullptr, FD_EINVAL, "space_order must be even in [2,16] (got %d)", space_order);
  const int64_t nmin = eq == FD_ACOUSTIC ? 2 : 1;
  int64_t npts = 1;
  for (int d = 0; d < ndim; ++d) {
    if (shape[d] < nmin || shape[d] > (1 << 20))
      return fail(nullptr, FD_EINVAL, "shape[%d] = %lld out of range", d, (long long)shape[d]);
    if (!(spacing[d] > 0.0) || !std::isfinite(spacing[d]))
      return fail(nullptr, FD_EINVAL, "spacing[%d] must be positive and finite", d);
    npts *= shape[d];
  }
  if (npts > ((int64_t)1 << 34)) return fail(nullptr, FD_EINVAL, "grid too large");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, FD_EINVAL, "dt must be positive and finite");
  fd_options o;
  fd_options_default(&o);
  if (opt) o = *opt;
  if (o.kernel < FD_KERNEL_AUTO || o.kernel > FD_KERNEL_TMA)
    return fail(nullptr, FD_EINVAL, "unknown kernel selector %d", o.kernel);
  if (o.boundary != FD_BOUNDARY_ZERO && o.boundary != FD_BOUNDARY_ODD)
    return fail(nullptr, FD_EINVAL, "unknown boundary mode %d", o.boundary);
  if (o.dirichlet_interior != 0 && o.dirichlet_interior != 1)
    return fail(nullptr, FD_EINVAL, "dirichlet_interior must be 0 or 1");
  if (o.boundary == FD_BOUNDARY_ODD) {
    if (eq != FD_DIFFUSION)
      return fail(nullptr, FD_EUNSUPPORTED, "FD_BOUNDARY_ODD is for FD_DIFFUSION");
    if (!o.dirichlet_interior)
      return fail(nullptr, FD_EINVAL, "FD_BOUNDARY_ODD mirrors about held boundary nodes "
                                      "(dirichlet_interior = 1)");
    for (int d = 0; d < ndim; ++d)
      if (shape[d] - 1 < space_order / 2)
        return fail(nullptr, FD_EINVAL,
                    "FD_BOUNDARY_ODD needs shape[%d] - 1 >= space_order/2 for the mirror", d);
  }
  const double S = lib_symbol(space_order);
  if (eq == FD_DIFFUSION) {
    if (!(o.nu > 0.0) || !std::isfinite(o.nu)) return fail(nullptr, FD_EINVAL, "nu must be positive");
    double lam = 0.0;
    for (int d = 0; d < ndim; ++d) lam += S / (spacing[d] * spacing[d]);
    if (o.nu * dt * lam > 2.0 * (1.0 + 1e-12))
      return fail(nullptr, FD_EINVAL,
                  "dt = %g exceeds the forward-Euler limit %g (nu dt sum S/h^2 <= 2)", dt,
                  2.0 / (o.nu * lam));
  }

  c = new (std::nothrow) fd_ctx();
  if (!c) return fail(nullptr, FD_ENOMEM, "host allocation failed");
  c->ndim = ndim;
  for (int d = 0; d < ndim; ++d) {
    c->shape[d] = shape[d];
    c->h[d] = spacing[d];
  }
  c->so = space_order;
  c->dt = dt;
  c->eq = eq;
  c->opt = o;
  c->nc = 1 << ndim;
  const int R = space_order / 2;
  Geom &g = c->g;
  if (ndim == 3) {
    g.n0 = (int)shape[0]; g.n1 = (int)shape[1]; g.n2 = (int)shape[2];
    g.R0 = R;
  } else {
    g.n0 = 1; g.n1 = (int)shape[0]; g.n2 = (int)shape[1];
    g.R0 = 0;
  }
  g.R = R;
  g.px = kHaloX + ((g.n2 + R + 31) / 32) * 32;
  g.py = g.n1 + 2 * R;
  g.plane = (int64_t)g.px * g.py;
  g.total = g.plane * (g.n0 + 2 * g.R0);
  g.hold = (eq == FD_DIFFUSION && o.dirichlet_interior) ? 1 : 0;

  // coefficients (axis mapping: user axis d -> internal axis d + 3 - ndim)
  double w[kMaxR + 1];
  lib_weights(space_order, w);
  const double scale = eq == FD_DIFFUSION ? o.nu * dt : 1.0;
  std::memset(&c->coef, 0, sizeof c->coef);
  for (int d = 0; d < ndim; ++d) {
    const int ax = d + 3 - ndim;
    const double s = scale / (spacing[d] * spacing[d]);
    for (int k = 1; k <= R; ++k) {
      c->coef.w[ax][k] = (float)(w[k] * s);
      c->coef.wp[ax][k] = make_float2(c->coef.w[ax][k], c->coef.w[ax][k]);
    }
  }
  // 2-D with equal spacing: the 2-D kernels take one weight per offset (plain_lap)
  c->coef.iso2 = ndim == 2 && spacing[0] == spacing[1] ? 1 : 0;
  select_kernel(c);

  auto bail = [&](fd_status st) {
    g_create_error = c->err;
    fd_destroy(c);
    return st;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    fail(c, FD_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    return bail(FD_ECUDA);
  }
  if (o.cuda_stream) {
    c->stream = (cudaStream_t)o.cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      fail(c, FD_ECUDA, "stream creation: %s", cudaGetErrorString(e));
      return bail(FD_ECUDA);
    }
    c->own_stream = true;
  }
  fd_status st = FD_OK;
  for (int b = 0; b < 2 && !st; ++b) st = dalloc(c, &c->u[b], (size_t)g.total);
  if (!st && eq == FD_ACOUSTIC) st = dalloc(c, &c->A, (size_t)g.total);
  if (!st && eq == FD_ACOUSTIC) st = dalloc(c, &c->C, (size_t)g.total);
  if (!st && eq == FD_ACOUSTIC) st = dalloc(c, &c->m_dense, (size_t)npts);
  if (!st && !o.device_ptrs) st = dalloc(c, &c->stage, (size_t)npts);
  if (!st) st = dalloc(c, &c->d_step, 1);
  if (!st) st = dalloc(c, &c->d_stats, 4);
  if (!st) st = dalloc(c, &c->d_err, 4);
  if (st) return bail(st);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    e = cudaMemsetAsync(c->u[b], 0, g.total * sizeof(float), c->stream);
  if (eq == FD_ACOUSTIC) {
    if (!e) e = cudaMemsetAsync(c->A, 0, g.total * sizeof(float), c->stream);
    if (!e) e = cudaMemsetAsync(c->C, 0, g.total * sizeof(float), c->stream);
  }
  if (!e) e = cudaMemsetAsync(c->d_err, 0, 4 * sizeof(int), c->stream);
  if (!e) e = cudaMemsetAsync(c->d_step, 0, sizeof(int64_t), c->stream);
  if (!e && !o.device_ptrs && eq == FD_ACOUSTIC) {
    e = cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&c->ev_model_free, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming);
    // the buffers were allocated and cleared on the context stream
    if (!e) e = cudaEventRecord(c->ev_model_free, c->stream);
  }
  if (e) {
    fail(c, FD_ECUDA, "initialisation: %s", cudaGetErrorString(e));
    return bail(FD_ECUDA);
  }
  // pipelined 3-D kernel where it applies
  c->use_tma = false;
  if (ndim == 3 && o.kernel != FD_KERNEL_PLAIN) {
    const char *why = nullptr;
    c->iso = spacing[0] == spacing[1] && spacing[1] == spacing[2];
    e = plan_tma(c->tma, c->g, eq == FD_ACOUSTIC ? kAcoustic : kDiffusion, c->iso, c->u, c->A,
                 c->C, 0, 0, 0, default_aligned(eq), &why, kTmaTX, ctx_origin(c));
    if (e == cudaSuccess) {
      c->use_tma = true;
      c->kernel_name = c->tma.name;
      if (o.autotune) {
        st = autotune_impl(c, 5, nullptr, nullptr, 0, nullptr);
        if (st) return bail(st);
      }
    } else {
      cudaGetLastError();
      if (o.kernel == FD_KERNEL_TMA) {
        fail(c, FD_EUNSUPPORTED, "TMA kernel unavailable: %s", why ? why : cudaGetErrorString(e));
        return bail(FD_EUNSUPPORTED);
      }
    }
  }
  *out = c;
  return FD_OK;
}

fd_status fd_set_model(fd_ctx *c, const float *m, const float *damp) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (c->eq != FD_ACOUSTIC) return fail(c, FD_EUNSUPPORTED, "fd_set_model is for FD_ACOUSTIC");
  if (!m) return fail(c, FD_EINVAL, "m is NULL");
  const size_t n = (size_t)c->g.n0 * c->g.n1 * c->g.n2;
  float *damp_dev = nullptr;
  if (c->opt.device_ptrs) {
    st = to_device(c, c->m_dense, m, n);
    if (st) return st;
    damp_dev = const_cast<float *>(damp);
  } else {
    // upload on the copy stream once the queued readers of m_dense and stage
    // have run (steps in flight do not read them); the coefficients follow in
    // stream order, after the steps queued before this call
    CU(cudaStreamWaitEvent(c->copy, c->ev_model_free, 0));
    CU(cudaMemcpyAsync(c->m_dense, m, n * sizeof(float), cudaMemcpyHostToDevice, c->copy));
    if (damp) {
      CU(cudaMemcpyAsync(c->stage, damp, n * sizeof(float), cudaMemcpyHostToDevice, c->copy));
      damp_dev = c->stage;
    }
    CU(cudaEventRecord(c->ev_copied, c->copy));
    CU(cudaStreamWaitEvent(c->stream, c->ev_copied, 0));
  }
  unsigned init[2] = {0x7f800000u, 0u};
  CU(cudaMemcpyAsync(c->d_stats, init, sizeof init, cudaMemcpyHostToDevice, c->stream));
  k_coefficients<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->m_dense, damp_dev, c->A, c->C,
                                                            c->g, c->dt, c->d_stats);
  CHECK_LAUNCH();
  st = model_readers_queued(c);
  if (st) return st;
  unsigned stats[2];
  CU(cudaMemcpyAsync(stats, c->d_stats, sizeof stats, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->model_set = false;
  if (stats[1]) return fail(c, FD_EINVAL, "m must be positive and finite, damp non-negative and finite");
  float mmin;
  std::memcpy(&mmin, &stats[0], sizeof mmin);
  double lam = 0.0;
  const double S = lib_symbol(c->so);
  for (int d = 0; d < c->ndim; ++d) lam += S / (c->h[d] * c->h[d]);
  const double dtmax = 2.0 * std::sqrt((double)mmin / lam);
  if (c->dt > dtmax * (1.0 + 1e-12))
    return fail(c, FD_EINVAL, "dt = %g exceeds the leapfrog limit %g for min(m) = %g", c->dt,
                dtmax, (double)mmin);
  c->model_set = true;
  c->src_dirty = c->nsrc > 0;
  c->unit_c_dirty = true;
  return FD_OK;
}

fd_status fd_set_field(fd_ctx *c, const float *u_cur, const float *u_prev) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (!u_cur) return fail(c, FD_EINVAL, "u_cur is NULL");
  // diffusion: the boundary values go to both levels
  if (c->eq == FD_DIFFUSION || !u_prev || u_prev == u_cur)
    return load_field(c, c->u[c->cur], u_cur, c->u[c->cur ^ 1]);
  st = load_field(c, c->u[c->cur], u_cur);
  if (!st) st = load_field(c, c->u[c->cur ^ 1], u_prev);
  return st;
}

fd_status fd_reset(fd_ctx *c) {
  fd_status st = check_usable(c);
  if (st) return st;
  const size_t bytes = (size_t)c->g.total * sizeof(float);
  CU(cudaMemsetAsync(c->u[0], 0, bytes, c->stream));
  CU(cudaMemsetAsync(c->u[1], 0, bytes, c->stream));
  c->step = 0;
  if (c->nrec > 0) {
    if (c->rec) CU(cudaMemsetAsync(c->rec, 0, (size_t)c->rec_cap * c->nrec * sizeof(float), c->stream));
    c->rec_rows = 0;
  }
  return FD_OK;
}

fd_status fd_set_sources(fd_ctx *c, int nsrc, const float *coords, int nt, const float *wavelets) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (c->eq != FD_ACOUSTIC) return fail(c, FD_EUNSUPPORTED, "sources need FD_ACOUSTIC");
  if (nsrc < 0 || nsrc > (1 << 22)) return fail(c, FD_EINVAL, "nsrc out of range");
  if (nsrc > 0 && (!coords || !wavelets || nt < 1)) return fail(c, FD_EINVAL, "coords/wavelets missing");
  std::vector<float> pts;
  st = coords_to_host(c, coords, (size_t)nsrc * c->ndim, pts);
  if (st) return st;
  const int n = nsrc * c->nc;
  std::vector<int64_t> off(n), dense(n);
  std::vector<double> w(n);
  for (int j = 0; j < nsrc; ++j)
    if (!corners(c, &pts[(size_t)j * c->ndim], &off[(size_t)j * c->nc], &dense[(size_t)j * c->nc],
                 &w[(size_t)j * c->nc]))
      return fail(c, FD_EINVAL, "source %d lies outside the grid", j);
  CU(cudaStreamSynchronize(c->stream));
  // The same counts as before (the next shot of a seismic acquisition): the buffers are
  // refilled in place, so the captured graphs, which hold their addresses, stay.
  if (nsrc == 0 || nsrc != c->nsrc || nt != c->nt_wav) {
    dfree(c, c->src_off); dfree(c, c->src_dense); dfree(c, c->src_w); dfree(c, c->src_scale); dfree(c, c->wav);
    drop_graphs(c);
    c->nsrc = 0;
    c->nt_wav = 0;
    c->h_src_dense.clear();
    c->sp_dirty = true;
    if (nsrc == 0) return FD_OK;
    if ((st = dalloc(c, &c->src_off, n)) || (st = dalloc(c, &c->src_dense, n)) ||
        (st = dalloc(c, &c->src_w, n)) || (st = dalloc(c, &c->src_scale, n)) ||
        (st = dalloc(c, &c->wav, (size_t)nt * nsrc)))
      return st;
  }
  // corners another slab owns: weight 0 at a valid node (their scale is 0)
  std::vector<int64_t> dense_dev(dense);
  for (int64_t &d : dense_dev) d = std::max<int64_t>(d, 0);
  CU(cudaMemcpyAsync(c->src_off, off.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->src_dense, dense_dev.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice,
                     c->stream));
  CU(cudaMemcpyAsync(c->src_w, w.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  st = to_device(c, c->wav, wavelets, (size_t)nt * nsrc);
  if (st) return st;
  CU(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
  c->nsrc = nsrc;
  c->nt_wav = nt;
  c->src_dirty = true;
  c->h_src_dense = dense;
  c->sp_dirty = true;
  return FD_OK;
}

fd_status fd_set_receivers(fd_ctx *c, int nrec, const float *coords) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (c->eq != FD_ACOUSTIC) return fail(c, FD_EUNSUPPORTED, "receivers need FD_ACOUSTIC");
  if (nrec < 0 || nrec > (1 << 22)) return fail(c, FD_EINVAL, "nrec out of range");
  if (nrec > 0 && !coords) return fail(c, FD_EINVAL, "coords missing");
  std::vector<float> pts;
  st = coords_to_host(c, coords, (size_t)nrec * c->ndim, pts);
  if (st) return st;
  const int n = nrec * c->nc;
  std::vector<int64_t> off(n), dense(n);
  std::vector<double> w(n);
  std::vector<float> wf(n);
  for (int k = 0; k < nrec; ++k)
    if (!corners(c, &pts[(size_t)k * c->ndim], &off[(size_t)k * c->nc], &dense[(size_t)k * c->nc],
                 &w[(size_t)k * c->nc]))
      return fail(c, FD_EINVAL, "receiver %d lies outside the grid", k);
  for (int i = 0; i < n; ++i) wf[i] = (float)w[i];
  CU(cudaStreamSynchronize(c->stream));
  if (nrec > 0 && nrec == c->nrec) {
    // same count: refill in place and keep the (cleared) trace buffer, so the
    // captured graphs stay valid
    if (c->rec)
      CU(cudaMemsetAsync(c->rec, 0, (size_t)c->rec_cap * nrec * sizeof(float), c->stream));
    c->rec_rows = 0;
  } else {
    dfree(c, c->rec_off); dfree(c, c->rec_w); dfree(c, c->rec);
    drop_graphs(c);
    c->nrec = 0;
    c->rec_cap = 0;
    c->rec_rows = 0;
    if (nrec == 0) return FD_OK;
    if ((st = dalloc(c, &c->rec_off, n)) || (st = dalloc(c, &c->rec_w, n))) return st;
  }
  CU(cudaMemcpyAsync(c->rec_off, off.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->rec_w, wf.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->nrec = nrec;
  if (c->step > 0) {  // rows before the current step stay zero
    st = ensure_rec_capacity(c, c->step + 1);
    if (st) return st;
    c->rec_rows = c->step + 1;
  }
  return FD_OK;
}

}  // extern "C"

namespace {

// The time loop: nt steps from the current state, by graph replay (graphs)
// or by launching each step.
fd_status run_steps(fd_ctx *c, int nt, bool graphs) {
  fd_status st = FD_OK;
  if (c->eq == FD_ACOUSTIC && !c->model_set)
    return fail(c, FD_ESTATE, "fd_set_model has not succeeded");
  if (c->nsrc > 0 && c->step + nt > c->nt_wav)
    return fail(c, FD_EINVAL, "step %lld exceeds the wavelet length %d",
                (long long)(c->step + nt), c->nt_wav);
  if (nt == 0) return FD_OK;
  if (c->nrec > 0) {
    st = ensure_rec_capacity(c, c->step + nt + 1);
    if (st) return st;
  }
  st = prepare_sources(c);
  if (st) return st;
  const bool was_fused = c->fused;
  st = prepare_fused(c);
  if (st) return st;
  if (was_fused != c->fused) drop_graphs(c);
  st = prepare_unit_c(c);
  if (st) return st;
  k_set_step<<<1, 1, 0, c->stream>>>(c->d_step, c->step);
  CHECK_LAUNCH();
  if (c->nrec > 0 && c->rec_rows == 0 && c->step == 0) {
    st = launch_interp_row0(c);
    if (st) return st;
  }
  for (int done = 0; done < nt;) {
    const int len = std::min(kGraphChunk, nt - done);
    if (c->fwi_seq_on) c->fwi_seq.i0 = done;
    if (graphs && c->opt.use_graphs) {
      cudaGraphExec_t exec;
      int64_t kernels = 0;
      st = get_graph(c, c->cur, len, &exec, &kernels);
      if (st) return st;
      // profile mode: the replayed chunk is timed as a whole (its len stencil
      // launches and the gaps between them)
      if (c->opt.profile && (st = profile_mark(c, false, 0))) return st;
      CU(cudaGraphLaunch(exec, c->stream));
      if (c->opt.profile && (st = profile_mark(c, true, len))) return st;
      c->launches += kernels;
    } else {
      st = enqueue_chunk(c, c->cur, len, c->opt.profile != 0);
      if (st) return st;
    }
    c->cur ^= (chunk_flips(c, len) & 1);
    done += len;
  }
  c->step += nt;
  if (c->nrec > 0) c->rec_rows = c->step + 1;
  return FD_OK;
}

}  // namespace

extern "C" {

fd_status fd_run(fd_ctx *c, int nt) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (nt < 0) return fail(c, FD_EINVAL, "nt must be >= 0");
  return run_steps(c, nt, true);
}

fd_status fd_step_fwi(fd_ctx *c, float *d2_out, float *img_g, const float *img_d2, double scale) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (c->eq != FD_ACOUSTIC || !c->use_tma || !c->tma.fn_fwi)
    return fail(c, FD_EUNSUPPORTED,
                "fd_step_fwi needs the pipelined 3-D acoustic kernel with 32-wide tiles");
  if (img_g && !img_d2) return fail(c, FD_EINVAL, "img_g needs img_d2");
  c->fwi_d2 = d2_out;
  c->fwi_img = img_g;
  c->fwi_img_d2 = img_d2;
  c->fwi_scale = (float)scale;
  c->fwi_on = true;
  st = run_steps(c, 1, false);
  c->fwi_on = false;
  return st;
}

fd_status fd_run_fwi(fd_ctx *c, int nt, float *d2_base, const float *img_d2_base,
                     int64_t stride, int reverse, float *img_g, double scale) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (c->eq != FD_ACOUSTIC || !c->use_tma || !c->tma.fn_fwi)
    return fail(c, FD_EUNSUPPORTED,
                "fd_run_fwi needs the pipelined 3-D acoustic kernel with 32-wide tiles");
  if (nt < 0) return fail(c, FD_EINVAL, "nt must be >= 0");
  if (img_g && !img_d2_base) return fail(c, FD_EINVAL, "img_g needs img_d2_base");
  if ((d2_base || img_d2_base) && stride < c->g.total)
    return fail(c, FD_EINVAL, "stride %lld is below fd_field_elems", (long long)stride);
  if (reverse != 0 && reverse != 1) return fail(c, FD_EINVAL, "reverse must be 0 or 1");
  FwiSeq q;
  q.d2_base = d2_base;
  q.img_d2_base = img_d2_base;
  q.img = img_g;
  q.stride = stride;
  q.nt = nt;
  q.reverse = reverse;
  q.scale = (float)scale;
  c->fwi_seq = q;
  c->fwi_seq_on = true;
  c->fwi_on = true;
  st = run_steps(c, nt, true);
  c->fwi_on = false;
  c->fwi_seq_on = false;
  return st;
}

fd_status fd_residual(fd_ctx *c, const float *d_obs, float *adj_wav, double *J) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (c->eq != FD_ACOUSTIC || c->nrec == 0 || c->rec_rows < 1)
    return fail(c, FD_ESTATE, "fd_residual needs recorded traces");
  if (!d_obs) return fail(c, FD_EINVAL, "d_obs is NULL");
  const int64_t rows = c->rec_rows, n = rows * c->nrec;
  constexpr int kBlocks = 512, kThreads = 256;
  if (!c->fwi_partial && (st = dalloc(c, &c->fwi_partial, kBlocks + 1))) return st;
  k_residual<<<kBlocks, kThreads, 0, c->stream>>>(c->rec, d_obs, adj_wav, rows, c->nrec,
                                                  c->fwi_partial);
  CHECK_LAUNCH();
  k_sum_partials<<<1, kThreads, 0, c->stream>>>(c->fwi_partial, kBlocks, c->fwi_partial + kBlocks);
  CHECK_LAUNCH();
  if (J) {
    CU(cudaMemcpyAsync(J, c->fwi_partial + kBlocks, sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  (void)n;
  return FD_OK;
}

fd_status fd_field_to_dense(fd_ctx *c, const float *padded, float *dense) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (!padded || !dense) return fail(c, FD_EINVAL, "NULL field");
  const int64_t n = (int64_t)c->g.n0 * c->g.n1 * c->g.n2;
  k_gather<<<blocks_for(n, 256), 256, 0, c->stream>>>(padded, dense, c->g);
  CHECK_LAUNCH();
  return FD_OK;
}

fd_status fd_read(fd_ctx *c, float *u, float *rec) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (u) {
    st = store_field(c, c->u[c->cur], u);
    if (st) return st;
  }
  if (rec && c->nrec > 0) {
    const int64_t rows = c->step + 1;
    if (c->rec_rows < rows) {
      // no step has been run since the receivers were set: record row 0 now
      st = ensure_rec_capacity(c, rows);
      if (st) return st;
      k_set_step<<<1, 1, 0, c->stream>>>(c->d_step, 0);
      CHECK_LAUNCH();
      st = launch_interp_row0(c);
      if (st) return st;
      c->rec_rows = 1;
    }
    CU(cudaMemcpyAsync(rec, c->rec, (size_t)rows * c->nrec * sizeof(float),
                       c->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
  }
  int errs[4];
  CU(cudaMemcpyAsync(errs, c->d_err, sizeof errs, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (errs[0])
    return fail(c, FD_ETIMEOUT, "a stencil kernel gave up waiting (code %d, block %d)", errs[0],
                errs[1]);
  return FD_OK;
}

fd_status fd_read_prev(fd_ctx *c, float *u_prev) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (!u_prev) return fail(c, FD_EINVAL, "u_prev is NULL");
  st = store_field(c, c->u[c->cur ^ 1], u_prev);
  if (st) return st;
  CU(cudaStreamSynchronize(c->stream));
  return FD_OK;
}

fd_status fd_set_step(fd_ctx *c, int64_t n) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (n < 0) return fail(c, FD_EINVAL, "step must be >= 0");
  c->step = n;
  if (c->nrec > 0) {
    st = ensure_rec_capacity(c, n + 1);
    if (st) return st;
    // n = 0: row 0 is recorded by the next fd_run; n > 0: rows 0..n keep
    // their contents (zero in a context that has not run)
    c->rec_rows = n == 0 ? 0 : n + 1;
  }
  return FD_OK;
}

int64_t fd_steps_done(const fd_ctx *c) { return c ? c->step : -1; }

fd_status fd_profile(fd_ctx *c, int64_t *launches, double *stencil_ms) {
  fd_status st = check_usable(c);
  if (st) return st;
  CU(cudaStreamSynchronize(c->stream));
  double total = 0.0;
  int64_t n = 0;
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    total += ms;
    n += c->ev_launches[i / 2];
  }
  if (launches) *launches = n;
  if (stencil_ms) *stencil_ms = total;
  c->ev_used = 0;
  return FD_OK;
}

fd_status fd_get_tile_config(const fd_ctx *c, fd_tile_config *cfg) {
  if (!c || !cfg) return FD_EINVAL;
  if (!c->use_tma) return FD_EUNSUPPORTED;
  tile_of(c, cfg);
  return FD_OK;
}

fd_status fd_set_tile_config(fd_ctx *c, const fd_tile_config *cfg) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (!cfg) return fail(c, FD_EINVAL, "cfg is NULL");
  if (!c->use_tma) return fail(c, FD_EUNSUPPORTED, "the plain kernel has no tile configuration");
  const int tx = cfg->tile_x ? cfg->tile_x : kTmaTX;
  if (!tma_tx_supported(tx, c->eq == FD_ACOUSTIC ? kAcoustic : kDiffusion) || cfg->tile_y % kTmaNW ||
      (cfg->tile_y != 0 && !tma_ny_supported(cfg->tile_y / kTmaNW)) || cfg->zblock < 0 ||
      cfg->ctas_per_sm < 0 || cfg->aligned < 0 || cfg->aligned > 2 ||
      (cfg->skip_c != 0 && cfg->skip_c != 1))
    return fail(c, FD_EINVAL,
                "tile configuration %dx%d, zblock %d, %d CTAs/SM, aligned %d, skip_c %d is not offered",
                cfg->tile_x, cfg->tile_y, cfg->zblock, cfg->ctas_per_sm, cfg->aligned, cfg->skip_c);
  return replan(c, cfg->tile_y / kTmaNW, cfg->ctas_per_sm, cfg->zblock, cfg->aligned, cfg->skip_c,
                tx);
}

fd_status fd_autotune(fd_ctx *c, int reps, fd_tile_config *best, fd_tile_config *tried,
                      int max_tried, int *ntried) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (reps < 1) return fail(c, FD_EINVAL, "reps must be >= 1");
  if (!c->use_tma) return fail(c, FD_EUNSUPPORTED, "the plain kernel has no tile configuration");
  return autotune_impl(c, reps, best, tried, max_tried, ntried);
}

fd_status fd_autotune_fwi(fd_ctx *c, int reps, fd_tile_config *best, fd_tile_config *tried,
                          int max_tried, int *ntried) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (reps < 1) return fail(c, FD_EINVAL, "reps must be >= 1");
  if (c->eq != FD_ACOUSTIC || !c->use_tma)
    return fail(c, FD_EUNSUPPORTED, "fd_autotune_fwi needs the pipelined 3-D acoustic kernel");
  return autotune_impl(c, reps, best, tried, max_tried, ntried, true);
}

const char *fd_kernel_name(const fd_ctx *c) { return c ? c->kernel_name : "none"; }

// ---------------------------------------------------------------------------
// z-slab sub-domains (one grid split along z; the paper's OPS backend leaves
// the distributed-memory partitioning of a structured block to the library,
// thesis §2.2).  Halo planes of the current level are refreshed from the
// neighbours' boundary planes after every step.
// ---------------------------------------------------------------------------
fd_status fd_set_subdomain(fd_ctx *c, int64_t z_origin, int64_t z_global) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (c->ndim != 3 || c->eq != FD_ACOUSTIC)
    return fail(c, FD_EUNSUPPORTED, "z-slab sub-domains are for 3-D FD_ACOUSTIC contexts");
  if (c->nsrc > 0 || c->nrec > 0)
    return fail(c, FD_ESTATE, "set the sub-domain before the sources and receivers");
  if (z_origin == 0 && z_global == 0) {
    const bool was = c->z_global > 0;
    c->z_origin = c->z_global = 0;
    if (was && c->use_tma)
      return replan(c, c->tma.ny, c->tma.per_sm, c->tma.args.zblock, c->tma.args.aligned,
                    c->skip_c ? 1 : 0, c->tma.tx);
    return FD_OK;
  }
  if (z_origin < 0 || z_global < 2 || z_origin + c->shape[0] > z_global)
    return fail(c, FD_EINVAL, "slab [%lld, %lld) does not fit a grid of %lld z nodes",
                (long long)z_origin, (long long)(z_origin + c->shape[0]), (long long)z_global);
  c->z_origin = z_origin;
  c->z_global = z_global;
  // the z halo now holds the neighbours' planes: the tensor maps read it from memory
  if (c->use_tma)
    return replan(c, c->tma.ny, c->tma.per_sm, c->tma.args.zblock, c->tma.args.aligned,
                  c->skip_c ? 1 : 0, c->tma.tx);
  return FD_OK;
}

int64_t fd_halo_elems(const fd_ctx *c) {
  return (c && c->ndim == 3) ? (int64_t)c->g.R * c->g.plane : -1;
}

namespace {
// Padded offset of the R planes a halo exchange reads (face: 0 = the first R
// interior planes, 1 = the last R) or writes (halo: 0 = below the interior, 1 = above).
int64_t face_offset(const fd_ctx *c, int side) {
  return side == 0 ? (int64_t)c->g.R * c->g.plane : (int64_t)c->g.n0 * c->g.plane;
}
int64_t halo_offset(const fd_ctx *c, int side) {
  return side == 0 ? 0 : (int64_t)(c->g.n0 + c->g.R) * c->g.plane;
}
fd_status halo_args_ok(fd_ctx *c, int side) {
  if (c->ndim != 3) return fail(c, FD_EUNSUPPORTED, "halo exchange is along z of a 3-D grid");
  if (side != 0 && side != 1) return fail(c, FD_EINVAL, "side must be 0 or 1");
  if (c->g.n0 < c->g.R)
    return fail(c, FD_EINVAL, "a slab of %d planes is thinner than the halo (%d)", c->g.n0, c->g.R);
  return FD_OK;
}
}  // namespace

fd_status fd_halo_export(fd_ctx *c, int side, float *dst) {
  fd_status st = check_usable(c);
  if (st) return st;
  if ((st = halo_args_ok(c, side))) return st;
  if (!dst) return fail(c, FD_EINVAL, "dst is NULL");
  CU(cudaMemcpyAsync(dst, c->u[c->cur] + face_offset(c, side),
                     (size_t)fd_halo_elems(c) * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  return FD_OK;
}

fd_status fd_halo_import(fd_ctx *c, int side, const float *src) {
  fd_status st = check_usable(c);
  if (st) return st;
  if ((st = halo_args_ok(c, side))) return st;
  if (!src) return fail(c, FD_EINVAL, "src is NULL");
  CU(cudaMemcpyAsync(c->u[c->cur] + halo_offset(c, side), src,
                     (size_t)fd_halo_elems(c) * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  return FD_OK;
}

fd_status fd_halo_copy(fd_ctx *dst, int side, fd_ctx *src) {
  fd_status st = check_usable(src);
  if (st) return st;
  if ((st = check_usable(dst))) return st;
  fd_ctx *c = dst;  // errors are reported on the receiving context
  if ((st = halo_args_ok(dst, side))) return st;
  if ((st = halo_args_ok(src, side ^ 1))) {
    dst->err = src->err;
    return st;
  }
  if (src->g.R != dst->g.R || src->g.plane != dst->g.plane || src->g.n1 != dst->g.n1 ||
      src->g.n2 != dst->g.n2)
    return fail(c, FD_EINVAL, "neighbouring slabs must share order and plane layout");
  // the lower halo takes the neighbour's last R planes, the upper its first R
  const size_t bytes = (size_t)fd_halo_elems(dst) * sizeof(float);
  float *to = dst->u[dst->cur] + halo_offset(dst, side);
  const float *from = src->u[src->cur] + face_offset(src, side ^ 1);
  const bool cross = src->stream != dst->stream;
  if (cross) {
    if (!src->ev_halo) {
      CU(cudaSetDevice(src->device));
      CU(cudaEventCreateWithFlags(&src->ev_halo, cudaEventDisableTiming));
      CU(cudaSetDevice(dst->device));
    }
    if (!dst->ev_halo) CU(cudaEventCreateWithFlags(&dst->ev_halo, cudaEventDisableTiming));
    CU(cudaEventRecord(src->ev_halo, src->stream));  // the neighbour's step is done
    CU(cudaStreamWaitEvent(dst->stream, src->ev_halo, 0));
  }
  if (src->device == dst->device)
    CU(cudaMemcpyAsync(to, from, bytes, cudaMemcpyDeviceToDevice, dst->stream));
  else
    CU(cudaMemcpyPeerAsync(to, dst->device, from, src->device, bytes, dst->stream));
  if (cross) {
    // the neighbour overwrites this level two steps on: after the copy
    CU(cudaEventRecord(dst->ev_halo, dst->stream));
    CU(cudaStreamWaitEvent(src->stream, dst->ev_halo, 0));
  }
  return FD_OK;
}

fd_status fd_run_slabs(fd_ctx *const *slabs, int nslabs, int nt) {
  if (!slabs || nslabs < 1 || nt < 0) return FD_EINVAL;
  for (int s = 0; s < nslabs; ++s) {
    fd_ctx *c = slabs[s];
    fd_status st = check_usable(c);
    if (st) return st;
    const int64_t want = s == 0 ? 0 : slabs[s - 1]->z_origin + slabs[s - 1]->shape[0];
    if (nslabs > 1 && (c->z_global == 0 || c->z_origin != want ||
                       c->z_global != slabs[0]->z_global ||
                       (s == nslabs - 1 && c->z_origin + c->shape[0] != c->z_global)))
      return fail(c, FD_EINVAL, "slab %d does not continue the z-slabs before it", s);
    if (c->step != slabs[0]->step) return fail(c, FD_ESTATE, "slabs are at different steps");
  }
  auto exchange = [&]() -> fd_status {
    for (int s = 0; s + 1 < nslabs; ++s) {
      fd_status st = fd_halo_copy(slabs[s + 1], 0, slabs[s]);
      if (!st) st = fd_halo_copy(slabs[s], 1, slabs[s + 1]);
      if (st) return st;
    }
    return FD_OK;
  };
  fd_status st = exchange();  // the current level's halos (after fd_set_field, fd_reset)
  for (int n = 0; n < nt && !st; ++n) {
    for (int s = 0; s < nslabs && !st; ++s) {
      fd_ctx *c = slabs[s];
      st = check_usable(c);
      if (!st) st = run_steps(c, 1, true);
    }
    if (!st) st = exchange();
  }
  return st;
}

fd_status fd_accumulate_traces(fd_ctx *c, float *acc) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (!acc) return fail(c, FD_EINVAL, "acc is NULL");
  const int64_t n = c->nrec > 0 ? c->rec_rows * c->nrec : 0;
  if (n == 0) return FD_OK;
  k_accumulate<<<blocks_for(n, 256), 256, 0, c->stream>>>(acc, c->rec, n);
  CHECK_LAUNCH();
  return FD_OK;
}

fd_status fd_skip_c_planes(fd_ctx *c, int64_t *flagged, int64_t *total) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (!flagged || !total) return fail(c, FD_EINVAL, "flagged/total is NULL");
  *flagged = 0;
  *total = 0;
  if (!c->use_tma || !c->skip_c || !c->model_set) return FD_OK;
  st = prepare_unit_c(c);
  if (st) return st;
  const size_t n = (size_t)c->tma.args.ntiles * c->g.n0;
  std::vector<unsigned char> h(n);
  CU(cudaMemcpyAsync(h.data(), c->unit_c, n, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  int64_t k = 0;
  for (unsigned char f : h) k += f ? 1 : 0;
  *flagged = k;
  *total = (int64_t)n;
  return FD_OK;
}

int64_t fd_field_elems(const fd_ctx *c) { return c ? c->g.total : -1; }

fd_status fd_snapshot(fd_ctx *c, float *dst_cur, float *dst_prev) {
  fd_status st = check_usable(c);
  if (st) return st;
  const size_t bytes = (size_t)c->g.total * sizeof(float);
  if (dst_cur) CU(cudaMemcpyAsync(dst_cur, c->u[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (dst_prev)
    CU(cudaMemcpyAsync(dst_prev, c->u[c->cur ^ 1], bytes, cudaMemcpyDeviceToDevice, c->stream));
  return FD_OK;
}

fd_status fd_restore(fd_ctx *c, const float *src_cur, const float *src_prev) {
  fd_status st = check_usable(c);
  if (st) return st;
  if (!src_cur || !src_prev) return fail(c, FD_EINVAL, "both levels are needed");
  const size_t bytes = (size_t)c->g.total * sizeof(float);
  CU(cudaMemcpyAsync(c->u[c->cur], src_cur, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(c->u[c->cur ^ 1], src_prev, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return FD_OK;
}

fd_status fd_imaging(fd_ctx *adj, float *g, const float *u_next, const float *u_cur,
                     const float *u_prev, double scale) {
  fd_ctx *c = adj;
  fd_status st = check_usable(c);
  if (st) return st;
  if (!g || !u_next || !u_cur || !u_prev) return fail(c, FD_EINVAL, "NULL field");
  const int64_t n = (int64_t)c->g.n0 * c->g.n1 * c->g.n2;
  k_imaging<<<blocks_for(n, 256), 256, 0, c->stream>>>(g, c->u[c->cur], u_next, u_cur, u_prev,
                                                        c->g, (float)scale);
  CHECK_LAUNCH();
  return FD_OK;
}

int64_t fd_kernel_launches(const fd_ctx *c) { return c ? c->launches : -1; }

void fd_destroy(fd_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  for (auto e : c->ev) cudaEventDestroy(e);
  destroy_tma(c->tma);
  dfree(c, c->u[0]); dfree(c, c->u[1]); dfree(c, c->A); dfree(c, c->C); dfree(c, c->m_dense); dfree(c, c->stage);
  dfree(c, c->d_step); dfree(c, c->d_stats); dfree(c, c->d_err);
  dfree(c, c->wav); dfree(c, c->src_scale); dfree(c, c->src_off); dfree(c, c->src_dense); dfree(c, c->src_w);
  dfree(c, c->rec_off); dfree(c, c->rec_w); dfree(c, c->rec);
  dfree(c, c->sp_entries); dfree(c, c->sp_first); dfree(c, c->unit_c); dfree(c, c->fwi_partial);
  for (int i = 0; i < 2; ++i) {
    if (c->ev_step[i]) cudaEventDestroy(c->ev_step[i]);
    if (c->ev_rec[i]) cudaEventDestroy(c->ev_rec[i]);
  }
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->copy) {
    cudaStreamSynchronize(c->copy);
    cudaStreamDestroy(c->copy);
  }
  if (c->ev_model_free) cudaEventDestroy(c->ev_model_free);
  if (c->ev_copied) cudaEventDestroy(c->ev_copied);
  if (c->ev_halo) cudaEventDestroy(c->ev_halo);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char *fd_last_error(const fd_ctx *c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

}  // extern "C"

namespace {

// Median µs of reps launches of plan p (after two warm-up launches), reading
// the context's current levels and writing `out`, without sources.
// With fwi, one repetition is a plain step, a step with the second-difference
// epilogue (into fwi_buf[0]) and a step with the imaging epilogue (reading
// fwi_buf[0], accumulating into fwi_buf[1]): the kernels of one backward step of
// the FWI sweep.
// Timed the way fd_run runs the step: reps repetitions captured in a CUDA graph and
// replayed kTuneBatches times with an event pair around each replay (eager batches of
// back-to-back launches where the stream cannot capture); the median replay, per
// repetition.  Launching with an event before every launch ranked the x-pair tile
// ahead of the 32-wide one at 256³ so 8, which replays 2-4 % faster in the step graphs.
constexpr int kTuneBatches = 3;
// The plan steps on two scratch levels (copies of the context's), rotating them like
// fd_run: each launch reads the level the previous one wrote, so the timing sees the
// L2 reuse of real steps (part of u^{n+1} is still in L2 when it is read as u^n).
fd_status time_plan(fd_ctx *c, const TmaPlan &p, int reps, cudaEvent_t *ev, double *us,
                    float *const *fwi_buf = nullptr, const unsigned char *unit_c = nullptr) {
  int cur = 0;
  reps += reps & 1;  // an even count: a replay ends on the parity it starts from
  auto step = [&](float *d2, float *img, const float *img_d2, float scale) -> cudaError_t {
    float *out = p.level[cur ^ 1];
    const cudaError_t e =
        (d2 || img) ? launch_tma_step_fwi(p, cur, out, c->coef, c->d_err, SparseArgs{}, d2, img,
                                          img_d2, scale, c->stream, unit_c)
                    : launch_tma_step(p, cur, out, c->coef, c->d_err, SparseArgs{}, c->stream,
                                      unit_c);
    cur ^= 1;
    return e;
  };
  auto one = [&]() -> fd_status {
    cudaError_t e = step(nullptr, nullptr, nullptr, 0.f);
    if (e == cudaSuccess && fwi_buf) e = step(fwi_buf[0], nullptr, nullptr, 0.f);
    if (e == cudaSuccess && fwi_buf) e = step(nullptr, fwi_buf[1], fwi_buf[0], 1.f);
    if (e != cudaSuccess) return fail(c, FD_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
    c->launches += fwi_buf ? 3 : 1;
    return FD_OK;
  };
  fd_status st = FD_OK;
  for (int i = 0; i < 2 && !st; ++i) st = one();  // warm-up
  if (st) return st;
  // capture the repetitions (launches counted when replayed)
  cudaGraphExec_t exec = nullptr;
  {
    cudaGraph_t graph = nullptr;
    const int64_t before = c->launches;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      for (int i = 0; i < reps && !st; ++i) st = one();
      const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
      if (!st && e == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
      if (st || e != cudaSuccess) exec = nullptr;
    }
    cudaGetLastError();  // a stream that cannot capture: eager batches below
    c->launches = before;
    if (st) return st;
  }
  const int64_t per_rep = fwi_buf ? 3 : 1;
  if (exec) CU(cudaGraphLaunch(exec, c->stream));  // the first replay uploads the graph
  for (int b = 0; b < kTuneBatches && !st; ++b) {
    CU(cudaEventRecord(ev[b], c->stream));
    if (exec) {
      CU(cudaGraphLaunch(exec, c->stream));
      c->launches += reps * per_rep;
    } else {
      for (int i = 0; i < reps && !st; ++i) st = one();
    }
  }
  if (st) {
    if (exec) cudaGraphExecDestroy(exec);
    return st;
  }
  CU(cudaEventRecord(ev[kTuneBatches], c->stream));
  CU(cudaEventSynchronize(ev[kTuneBatches]));
  std::vector<double> t(kTuneBatches);
  for (int b = 0; b < kTuneBatches; ++b) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, ev[b], ev[b + 1]));
    t[b] = 1e3 * ms / reps;
  }
  std::sort(t.begin(), t.end());
  *us = t[kTuneBatches / 2];
  if (exec) cudaGraphExecDestroy(exec);
  return FD_OK;
}

fd_status autotune_impl(fd_ctx *c, int reps, fd_tile_config *best, fd_tile_config *tried,
                        int max_tried, int *ntried, bool fwi) {
  if (ntried) *ntried = 0;
  const TuneKey key = tune_key(c, fwi);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && !tried) {
      const fd_tile_config cfg = it->second;
      fd_status st =
          replan(c, cfg.tile_y / kTmaNW, cfg.ctas_per_sm, cfg.zblock, cfg.aligned, cfg.skip_c,
                 cfg.tile_x);
      if (st) return st;
      c->tune_us = cfg.us_per_step;
      if (best) *best = cfg;
      return FD_OK;
    }
  }
  // two scratch levels (the plans step on copies of the current ones), and for the
  // FWI sweep the second-difference and imaging fields
  float *lev[2] = {nullptr, nullptr}, *fbuf[2] = {nullptr, nullptr};
  fd_status st = dalloc(c, &lev[0], (size_t)c->g.total);
  if (!st) st = dalloc(c, &lev[1], (size_t)c->g.total);
  if (!st)
    CU(cudaMemcpyAsync(lev[0], c->u[c->cur], c->g.total * sizeof(float),
                       cudaMemcpyDeviceToDevice, c->stream));
  if (!st)
    CU(cudaMemcpyAsync(lev[1], c->u[c->cur ^ 1], c->g.total * sizeof(float),
                       cudaMemcpyDeviceToDevice, c->stream));
  if (!st && fwi) st = dalloc(c, &fbuf[0], (size_t)c->g.total);
  if (!st && fwi) st = dalloc(c, &fbuf[1], (size_t)c->g.total);
  if (!st && fwi) CU(cudaMemsetAsync(fbuf[0], 0, c->g.total * sizeof(float), c->stream));
  if (!st && fwi) CU(cudaMemsetAsync(fbuf[1], 0, c->g.total * sizeof(float), c->stream));
  if (st) {
    dfree(c, lev[0]);
    dfree(c, lev[1]);
    dfree(c, fbuf[0]);
    dfree(c, fbuf[1]);
    return st;
  }
  std::vector<cudaEvent_t> ev(kTuneBatches + 1, nullptr);
  for (auto &e : ev)
    if (!st && cudaEventCreate(&e) != cudaSuccess) st = fail(c, FD_ECUDA, "event creation");
  const int eq = c->eq == FD_ACOUSTIC ? kAcoustic : kDiffusion;
  const int R = c->so / 2;
  const int zmin = std::min<int>(c->g.n0, std::max(8, 2 * R));
  // candidates: tile height × CTAs per SM × (equal tile-plane ranges with z-blocks of
  // share/2, share, 2·share | whole segments with z-blocks that make m or 2m
  // segments per tile, m = CTAs / tiles)
  struct Cand {
    int ny, cps, zb, aligned, tx;
  };
  std::vector<Cand> cands;
  // the x-pair kernel (tiles kXpTX wide) too, except for the FWI sweep (no FWI instance)
  const std::vector<int> widths =
      fwi ? std::vector<int>{kTmaTX} : std::vector<int>{kTmaTX, kXpTX};
  for (int tx : widths)
  for (int ny : {2, 3, 4}) {
    if (ny == 3 && (tx != kXpTX || !xp_hc_supported(R, 3))) continue;  // 24 rows: x-pair only
    TmaPlan p{};
    const char *why = nullptr;
    if (st || plan_tma(p, c->g, eq, c->iso, c->u, c->A, c->C, ny, 0, 0, 0, &why, tx,
                       ctx_origin(c)) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    for (int cps = 1; cps <= p.per_sm_max; ++cps) {
      TmaPlan q{};
      if (plan_tma(q, c->g, eq, c->iso, c->u, c->A, c->C, ny, cps, 0, 0, &why, tx,
                   ctx_origin(c)) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      const int share = q.args.zblock;
      cands.push_back({ny, cps, share, 0, tx});
      if (share / 2 > zmin) cands.push_back({ny, cps, share / 2, 0, tx});
      if (2 * share <= c->g.n0) cands.push_back({ny, cps, 2 * share, 0, tx});
      // segments no shorter than zmin planes
      const int mcap = std::max(1, c->g.n0 / zmin);
      const int m1 = std::max(1, (q.sms * cps) / q.args.ntiles);
      for (int m : {std::min(m1, mcap), std::min(2 * m1, mcap)}) {
        const int zb = (c->g.n0 + m - 1) / m;
        bool dup = false;
        for (const Cand &d : cands)
          dup |= d.ny == ny && d.cps == cps && d.zb == zb && d.aligned && d.tx == tx;
        if (!dup) cands.push_back({ny, cps, zb, 1, tx});
      }
      // work queue (x-pair tiles): z-layers thick first, thin last, taken by
      // whichever CTA is free
      if (tx == kXpTX) cands.push_back({ny, cps, 0, 2, tx});
    }
  }
  // each candidate once more skipping the C tiles where C = 1 (acoustic, R <= 4;
  // only with a model set: before it C is 0 everywhere and nothing would be skipped)
  const bool try_skip = c->eq == FD_ACOUSTIC && R <= 4 && c->model_set;
  unsigned char *flags = nullptr;
  // flags for the most tile-planes any candidate has (the smallest tile, kTmaTX × 16)
  const size_t max_flags = (size_t)((c->g.n2 + kTmaTX - 1) / kTmaTX) *
                           (size_t)((c->g.n1 + tma_ty(2) - 1) / tma_ty(2)) * c->g.n0;
  if (!st && try_skip) st = dalloc(c, &flags, max_flags);
  fd_tile_config win{};
  double win_us = 1e300;
  int n = 0;
  for (const Cand &cd : cands) {
    if (st) break;
    TmaPlan r{};
    const char *why = nullptr;
    if (plan_tma(r, c->g, eq, c->iso, lev, c->A, c->C, cd.ny, cd.cps, cd.zb, cd.aligned, &why,
                 cd.tx, ctx_origin(c)) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (fwi && !r.fn_fwi) continue;  // no FWI instance fits this grid
    for (int sk = 0; sk <= (try_skip ? 1 : 0) && !st; ++sk) {
      if (sk) {
        const int64_t nf = (int64_t)r.args.ntiles * c->g.n0;
        if ((size_t)nf > max_flags) {  // cannot happen: the smallest tile bounds the count
          st = fail(c, FD_ECUDA, "autotune: flag buffer too small");
          break;
        }
        k_unit_c<<<(unsigned)nf, 128, 0, c->stream>>>(c->C, c->g, r.args.tiles_x, cd.tx,
                                                       tma_ty(cd.ny), flags);
        if (cudaGetLastError() != cudaSuccess) {
          st = fail(c, FD_ECUDA, "autotune: flags kernel");
          break;
        }
      }
      double us = 0.0;
      st = time_plan(c, r, reps, ev.data(), &us, fwi ? fbuf : nullptr,
                     sk ? flags : nullptr);
      if (st) break;
      fd_tile_config cfg{cd.tx, tma_ty(cd.ny), r.args.zblock, r.per_sm, cd.aligned, sk, us};
      if (tried && n < max_tried) tried[n] = cfg;
      ++n;
      if (us < win_us) {
        win_us = us;
        win = cfg;
      }
    }
  }
  dfree(c, flags);
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  dfree(c, lev[0]);
  dfree(c, lev[1]);
  dfree(c, fbuf[0]);
  dfree(c, fbuf[1]);
  if (st) return st;
  // a candidate that gave up on a wait leaves its code in the error word
  int err[2] = {0, 0};
  CU(cudaMemcpyAsync(err, c->d_err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (err[0]) return fail(c, FD_ETIMEOUT, "autotune: pipelined kernel wait expired (code %d)", err[0]);
  if (n == 0) return fail(c, FD_EUNSUPPORTED, "autotune: no tile configuration could be planned");
  if (ntried) *ntried = n;
  st = replan(c, win.tile_y / kTmaNW, win.ctas_per_sm, win.zblock, win.aligned, win.skip_c,
              win.tile_x);
  if (st) return st;
  c->tune_us = win.us_per_step;
  if (best) *best = win;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = win;
  return FD_OK;
}

}  // namespace

// ===========================================================================
// Batches: many acoustic shots stepped together (continuous batching).
//
// Members stay ordinary contexts (their own fields, traces and step counters);
// a batch tick launches one persistent pipelined kernel for all 3-D members
// (k_stencil3d_tma<..., MULTI>: the CTAs share out the members' tile-planes),
// one kernel for all 2-D members, one injection kernel for the 2-D members'
// sources (3-D injection is fused), and one receiver kernel for everyone.
// ===========================================================================
struct fd_batch {
  int so = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<fd_ctx *> members;
  ShotDesc *d_shots = nullptr;   // 3-D members
  int4 *d_items = nullptr;       // work items of the pipelined kernel
  unsigned *d_ticket = nullptr;  // [2] item tickets
  size_t cap_items = 0;
  MemberDesc *d_mem = nullptr;   // every member (2-D stencil, injection, receivers)
  int2 *d_src = nullptr, *d_rec = nullptr;
  int64_t *d_tick = nullptr;
  size_t cap_shots = 0, cap_mem = 0, cap_src = 0, cap_rec = 0;
  std::vector<ShotDesc> h_shots;  // staging (pageable: cudaMemcpyAsync copies it out before
  std::vector<MemberDesc> h_mem;  // returning, so the next run may refill it at once)
  std::vector<int2> h_src, h_rec;
  std::vector<int4> h_items;
  cudaEvent_t ev = nullptr;
  // receivers of tick j on a side stream, overlapping tick j+1; tick j+2 (which
  // overwrites the level they read) waits for them
  cudaStream_t side = nullptr;
  cudaEvent_t ev_step[2] = {nullptr, nullptr}, ev_rec[2] = {nullptr, nullptr};
  // captured chunks of ticks, valid while the launch parameters are unchanged
  struct Graph {
    int len;
    int64_t kernels;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  std::vector<int64_t> graph_sig;
  std::vector<int> seen_len;  // chunk lengths launched once with graph_sig
  int64_t launches = 0;
  bool failed = false;
  std::string err;
};

namespace {

fd_status bfail(fd_batch *b, fd_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  b->err = buf;
  if (st == FD_ECUDA) b->failed = true;
  return st;
}

#define BCU(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? FD_ENOMEM : FD_ECUDA,          \
                   "%s failed: %s", #call, cudaGetErrorString(e_));                    \
  } while (0)

template <typename T>
fd_status bgrow(fd_batch *b, T **dev, T **host, size_t *cap, size_t need) {
  if (need <= *cap) return FD_OK;
  const size_t n = std::max<size_t>(need, 2 * *cap + 8);
  if (*dev) BCU(cudaStreamSynchronize(b->stream));  // earlier runs may still read it
  if (*dev) cudaFree(*dev);
  *dev = nullptr;
  BCU(cudaMalloc((void **)dev, n * sizeof(T)));
  if (host) {
    if (*host) cudaFreeHost(*host);
    *host = nullptr;
    BCU(cudaMallocHost((void **)host, n * sizeof(T)));
  }
  *cap = n;
  return FD_OK;
}

StencilFn2D batch2d_fn(int R) {
  switch (R) {
    case 1: return k_stencil2d_batch<1>;
    case 2: return k_stencil2d_batch<2>;
    case 3: return k_stencil2d_batch<3>;
    case 4: return k_stencil2d_batch<4>;
    case 5: return k_stencil2d_batch<5>;
    case 6: return k_stencil2d_batch<6>;
    case 7: return k_stencil2d_batch<7>;
    default: return k_stencil2d_batch<8>;
  }
}

}  // namespace

extern "C" {

fd_status fd_batch_create(fd_batch **out, int space_order, void *cuda_stream) {
  if (!out) return FD_EINVAL;
  *out = nullptr;
  if (space_order < 2 || space_order > 2 * kMaxR || (space_order & 1))
    return fail(nullptr, FD_EINVAL, "space_order must be even in [2,16] (got %d)", space_order);
  fd_batch *b = new (std::nothrow) fd_batch();
  if (!b) return fail(nullptr, FD_ENOMEM, "host allocation failed");
  b->so = space_order;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      b->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_tick, sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_ticket, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fail(nullptr, FD_ECUDA, "batch creation: %s", cudaGetErrorString(e));
    fd_batch_destroy(b);
    return FD_ECUDA;
  }
  *out = b;
  return FD_OK;
}

fd_status fd_batch_add(fd_batch *b, fd_ctx *c) {
  if (!b || !c) return FD_EINVAL;
  if (b->failed) return FD_ECUDA;
  if (c->failed) return bfail(b, FD_ECUDA, "member context has failed");
  if (c->eq != FD_ACOUSTIC || c->so != b->so)
    return bfail(b, FD_EINVAL, "members must be FD_ACOUSTIC contexts of space order %d", b->so);
  if (!c->model_set) return bfail(b, FD_ESTATE, "member has no model (fd_set_model)");
  if (c->ndim == 3 && !c->use_tma)
    return bfail(b, FD_EUNSUPPORTED, "3-D members need the pipelined kernel (FD_KERNEL_AUTO/TMA)");
  if (c->z_global > 0)
    return bfail(b, FD_EUNSUPPORTED, "z-slab sub-domains exchange halos (fd_run_slabs), not batches");
  if (c->device != b->device) return bfail(b, FD_EINVAL, "member lives on another device");
  if (std::find(b->members.begin(), b->members.end(), c) != b->members.end())
    return bfail(b, FD_EINVAL, "already a member");
  if (c->ndim == 3 && c->tma.tx != kTmaTX) {
    // the batched kernel has 32-wide tiles only: back to the default configuration
    fd_status st = replan(c, 0, 0, 0, default_aligned(c->eq));
    if (st) return bfail(b, st, "member replan: %s", c->err.c_str());
  }
  if (c->ndim == 3 && !b->members.empty()) {
    for (fd_ctx *o : b->members)
      if (o->ndim == 3 && (o->tma.fn_multi != c->tma.fn_multi ||
                           std::memcmp(o->coef.wp, c->coef.wp, sizeof c->coef.wp) != 0))
        return bfail(b, FD_EUNSUPPORTED, "3-D members must share their grid spacing");
  }
  b->members.push_back(c);
  return FD_OK;
}

fd_status fd_batch_remove(fd_batch *b, fd_ctx *c) {
  if (!b || !c) return FD_EINVAL;
  auto it = std::find(b->members.begin(), b->members.end(), c);
  if (it == b->members.end()) return bfail(b, FD_EINVAL, "not a member");
  // no wait: the member's stream already waits for the batch's last run, and the
  // next run rewrites the device tables in stream order
  b->members.erase(it);
  return FD_OK;
}

int fd_batch_size(const fd_batch *b) { return b ? (int)b->members.size() : -1; }

int64_t fd_batch_kernel_launches(const fd_batch *b) { return b ? b->launches : -1; }

const char *fd_batch_last_error(const fd_batch *b) { return b ? b->err.c_str() : ""; }

fd_status fd_batch_run(fd_batch *b, int nticks) {
  if (!b) return FD_EINVAL;
  if (b->failed) return FD_ECUDA;
  if (nticks < 0) return bfail(b, FD_EINVAL, "nticks must be >= 0");
  if (nticks == 0 || b->members.empty()) return FD_OK;
  BCU(cudaSetDevice(b->device));
  const int R = b->so / 2;
  // members: checks, per-member preparation, order after their own streams
  for (fd_ctx *c : b->members) {
    if (c->failed) return bfail(b, FD_ECUDA, "member context has failed");
    if (c->nsrc > 0 && c->step + nticks > c->nt_wav)
      return bfail(b, FD_EINVAL, "a member would pass its wavelet length");
    fd_status st = FD_OK;
    // the batched kernel runs the default tile: a tuned member goes back to it
    if (c->ndim == 3 && (c->tma.ny != tma_ny(R) || c->tma.tx != kTmaTX))
      st = replan(c, 0, 0, 0, default_aligned(c->eq));
    if (!st && c->nrec > 0) st = ensure_rec_capacity(c, c->step + nticks + 1);
    if (!st) st = prepare_sources(c);
    if (!st && c->ndim == 3) st = prepare_fused(c);
    if (st) return bfail(b, st, "member preparation: %s", c->err.c_str());
    if (c->nrec > 0 && c->rec_rows == 0 && c->step == 0) {  // trace row 0
      k_set_step<<<1, 1, 0, c->stream>>>(c->d_step, 0);
      st = launch_interp_row0(c);
      if (st) return bfail(b, st, "member trace row 0: %s", c->err.c_str());
      c->rec_rows = 1;
    }
    if (c->stream != b->stream) {
      BCU(cudaEventRecord(b->ev, c->stream));
      BCU(cudaStreamWaitEvent(b->stream, b->ev, 0));
    }
  }
  // descriptor tables (device tables are rewritten in stream order)
  std::vector<fd_ctx *> m3;
  for (fd_ctx *c : b->members)
    if (c->ndim == 3) m3.push_back(c);
  const size_t nm = b->members.size(), n3 = m3.size();
  fd_status st = bgrow<MemberDesc>(b, &b->d_mem, nullptr, &b->cap_mem, nm);
  if (!st) st = bgrow<ShotDesc>(b, &b->d_shots, nullptr, &b->cap_shots, std::max<size_t>(n3, 1));
  if (st) return st;
  b->h_mem.resize(nm);
  b->h_shots.resize(std::max<size_t>(n3, 1));
  b->h_src.clear();
  b->h_rec.clear();
  int64_t blk = 0;
  for (size_t i = 0; i < nm; ++i) {
    fd_ctx *c = b->members[i];
    MemberDesc &d = b->h_mem[i];
    std::memset(&d, 0, sizeof d);
    d.level[0] = c->u[0];
    d.level[1] = c->u[1];
    d.A = c->A;
    d.C = c->C;
    d.g = c->g;
    d.c = c->coef;
    d.cur0 = c->cur;
    d.step0 = c->step;
    d.src_off = c->src_off;
    d.src_scale = c->src_scale;
    d.wav = c->wav;
    d.nsrc = c->nsrc;
    d.nc = c->nc;
    d.rec_off = c->rec_off;
    d.rec_w = c->rec_w;
    d.rec = c->rec;
    d.nrec = c->nrec;
    d.blk0 = blk;  // non-decreasing over members; 3-D members own no 2-D blocks
    if (c->ndim == 2) {
      d.blocks_x = (c->g.n2 + 31) / 32;
      blk += (int64_t)d.blocks_x * ((c->g.n1 + 7) / 8);
      for (int k = 0; k < c->nsrc * c->nc; ++k) b->h_src.push_back(make_int2((int)i, k));
    }
    for (int k = 0; k < c->nrec; ++k) b->h_rec.push_back(make_int2((int)i, k));
  }
  // work items {shot, tile, za, zb}, z-layer by z-layer over all 3-D members,
  // tile by tile within a shot, so that CTAs taking consecutive tickets hold
  // neighbouring tiles at the same depth.  A batch whose work is at most 128
  // planes per CTA is cut into at most one item per CTA (each shot into layers
  // of about the average share, at least max(8, 2R) planes); a larger batch
  // into layers that are thick while much work remains and thinner towards the
  // end (guided), so the last items are short.
  const TmaPlan &plan0 = n3 ? m3[0]->tma : TmaPlan();
  b->h_items.clear();
  int grid3 = 0;
  if (n3) {
    const int G = std::max(plan0.grid_multi, 1);
    const int zmin = std::max(8, 2 * R);
    int64_t W = 0;
    int zmax = 0;
    for (fd_ctx *c : m3) {
      W += (int64_t)c->tma.args.ntiles * c->g.n0;
      zmax = std::max(zmax, c->g.n0);
    }
    const int64_t share = W / G;
    if (share <= 128) {
      // shot i gets floor(n0_i G / W) layers (so there are no more items than
      // CTAs), none thinner than zmin planes
      std::vector<int> height(n3), layers(n3);
      int kmax = 0;
      for (size_t i = 0; i < n3; ++i) {
        const int n0 = m3[i]->g.n0;
        const int64_t fit = (int64_t)n0 * G / std::max<int64_t>(W, 1);
        layers[i] = (int)std::max<int64_t>(1, std::min<int64_t>(n0 / zmin, fit));
        height[i] = (n0 + layers[i] - 1) / layers[i];
        kmax = std::max(kmax, layers[i]);
      }
      for (int k = 0; k < kmax; ++k)
        for (size_t i = 0; i < n3; ++i) {
          const int za = k * height[i];
          if (za >= m3[i]->g.n0) continue;
          const int zb = std::min(m3[i]->g.n0, za + height[i]);
          for (int t = 0; t < m3[i]->tma.args.ntiles; ++t)
            b->h_items.push_back(make_int4((int)i, t, za, zb));
        }
    } else {
      for (int z = 0; z < zmax;) {
        int64_t tiles_here = 0, rem = 0;
        for (fd_ctx *c : m3)
          if (c->g.n0 > z) {
            tiles_here += c->tma.args.ntiles;
            rem += (int64_t)c->tma.args.ntiles * (c->g.n0 - z);
          }
        // layer height: half a tile's remaining depth, no more than makes the
        // remaining work about two items per CTA, between 16 and 128 planes
        const int64_t per_tile = rem / std::max<int64_t>(tiles_here, 1);
        const int64_t fill = rem / (2 * (int64_t)G);
        const int h =
            (int)std::min<int64_t>(128, std::max<int64_t>(16, std::min(per_tile / 2, fill)));
        for (size_t i = 0; i < n3; ++i) {
          fd_ctx *c = m3[i];
          if (c->g.n0 <= z) continue;
          const int zb = std::min(c->g.n0, z + h);
          for (int t = 0; t < c->tma.args.ntiles; ++t)
            b->h_items.push_back(make_int4((int)i, t, z, zb));
        }
        z += h;
      }
    }
    grid3 = (int)std::min<int64_t>(plan0.grid_multi, (int64_t)b->h_items.size());
  }
  for (size_t i = 0; i < n3; ++i) {
    fd_ctx *c = m3[i];
    ShotDesc &d = b->h_shots[i];
    std::memset(&d, 0, sizeof d);
    d.map_u[0] = c->tma.map_u[0];
    d.map_u[1] = c->tma.map_u[1];
    d.map_t[0] = c->tma.map_t[0];
    d.map_t[1] = c->tma.map_t[1];
    d.map_a = c->tma.map_a;
    d.map_c = c->tma.map_c;
    d.org = c->tma.args.org;
    d.g = c->g;
    d.c = c->coef;
    d.level[0] = c->u[0];
    d.level[1] = c->u[1];
    d.tiles_x = c->tma.args.tiles_x;
    d.ntiles = c->tma.args.ntiles;
    d.zblock = c->g.n0;
    d.cur0 = c->cur;
    d.step0 = c->step;
    if (c->nsrc > 0) {
      d.entries = c->sp_entries;
      d.first = c->sp_first;
      d.src_scale = c->src_scale;
      d.wav = c->wav;
      d.nsrc = c->nsrc;
      d.nc = c->nc;
    }
  }
  if (!b->h_items.empty())
    st = bgrow<int4>(b, &b->d_items, nullptr, &b->cap_items, b->h_items.size());
  if (!st && !b->h_src.empty()) st = bgrow<int2>(b, &b->d_src, nullptr, &b->cap_src, b->h_src.size());
  if (!st && !b->h_rec.empty()) st = bgrow<int2>(b, &b->d_rec, nullptr, &b->cap_rec, b->h_rec.size());
  if (st) return st;
  BCU(cudaMemcpyAsync(b->d_mem, b->h_mem.data(), nm * sizeof(MemberDesc), cudaMemcpyHostToDevice,
                      b->stream));
  if (n3) {
    BCU(cudaMemcpyAsync(b->d_shots, b->h_shots.data(), n3 * sizeof(ShotDesc),
                        cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_items, b->h_items.data(), b->h_items.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemsetAsync(b->d_ticket, 0, 2 * sizeof(unsigned), b->stream));
  }
  if (!b->h_src.empty())
    BCU(cudaMemcpyAsync(b->d_src, b->h_src.data(), b->h_src.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  if (!b->h_rec.empty())
    BCU(cudaMemcpyAsync(b->d_rec, b->h_rec.data(), b->h_rec.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  k_set_step<<<1, 1, 0, b->stream>>>(b->d_tick, 0);
  BCU(cudaGetLastError());
  ++b->launches;
  // error word of the pipelined kernel: the first 3-D member's
  const int nsrc_e = (int)b->h_src.size(), nrec_e = (int)b->h_rec.size();
  const StencilFn2D f2 = batch2d_fn(R);
  int *const err3 = n3 ? m3[0]->d_err : nullptr;
  // the 3-D shots share their weights (fd_batch_add): a kernel parameter
  BatchArgs bargs{};
  bargs.shots = b->d_shots;
  bargs.items = b->d_items;
  bargs.nitems = (int)b->h_items.size();
  bargs.ticket = b->d_ticket;
  bargs.tick = b->d_tick;
  bargs.err = err3;
  if (n3) std::memcpy(bargs.wp, m3[0]->coef.wp, sizeof bargs.wp);
  // the kernels of `len` ticks (tick *d_tick + j, j < len), then the counter moves
  if (nrec_e && !b->side) {
    BCU(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      BCU(cudaEventCreateWithFlags(&b->ev_step[i], cudaEventDisableTiming));
      BCU(cudaEventCreateWithFlags(&b->ev_rec[i], cudaEventDisableTiming));
    }
  }
  auto enqueue = [&](int len, int64_t *kernels) -> cudaError_t {
    int64_t k = 0;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < len && e == cudaSuccess; ++j) {
      // tick j overwrites the level tick j-2's receivers read
      if (nrec_e && j >= 2) e = cudaStreamWaitEvent(b->stream, b->ev_rec[j & 1], 0);
      if (n3) {
        BatchArgs ba = bargs;
        ba.j = j;
        plan0.fn_multi<<<grid3, kTmaThreads, plan0.smem_multi, b->stream>>>(
            plan0.map_u[0], plan0.map_t[0], plan0.map_a, plan0.map_c, plan0.map_c, plan0.map_c,
            TmaArgs{}, ba);
        ++k;
      }
      if (blk > 0) {
        f2<<<(unsigned)blk, dim3(32, 8), 0, b->stream>>>(b->d_mem, (int)nm, b->d_tick, j);
        ++k;
      }
      if (nsrc_e) {
        k_inject_batch<<<(nsrc_e + 255) / 256, 256, 0, b->stream>>>(b->d_src, nsrc_e, b->d_mem,
                                                                    b->d_tick, j);
        ++k;
      }
      if (nrec_e) {  // on the side stream, after this tick's stencils and injection
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_step[j & 1], b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_step[j & 1], 0);
        k_interp_batch<<<(nrec_e * 8 + 255) / 256, 256, 0, b->side>>>(b->d_rec, nrec_e,
                                                                      b->d_mem, b->d_tick, j);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_rec[j & 1], b->side);
        ++k;
      }
    }
    if (nrec_e && e == cudaSuccess) {  // join the side stream before the tick counter moves
      e = cudaStreamWaitEvent(b->stream, b->ev_rec[(len - 1) & 1], 0);
      if (e == cudaSuccess && len >= 2) e = cudaStreamWaitEvent(b->stream, b->ev_rec[len & 1], 0);
    }
    if (e != cudaSuccess) return e;
    k_advance_step<<<1, 1, 0, b->stream>>>(b->d_tick, len);
    *kernels = k + 1;
    return cudaGetLastError();
  };
  // chunks of ticks replayed from captured graphs, keyed by everything a launch
  // takes as a parameter (tables are rewritten in place, so pointers repeat)
  const std::vector<int64_t> sig = {
      (int64_t)nm, (int64_t)n3, (int64_t)b->h_items.size(), grid3, blk, nsrc_e, nrec_e,
      (int64_t)(uintptr_t)b->d_shots, (int64_t)(uintptr_t)b->d_items,
      (int64_t)(uintptr_t)b->d_mem, (int64_t)(uintptr_t)b->d_src, (int64_t)(uintptr_t)b->d_rec,
      (int64_t)(uintptr_t)(n3 ? (void *)plan0.fn_multi : nullptr), plan0.smem_multi,
      (int64_t)(uintptr_t)err3,
      (int64_t)std::hash<std::string>()(
          std::string(reinterpret_cast<const char *>(bargs.wp), sizeof bargs.wp))};
  if (sig != b->graph_sig) {
    for (auto &gph : b->graphs) cudaGraphExecDestroy(gph.exec);
    b->graphs.clear();
    b->seen_len.clear();
    b->graph_sig = sig;
  }
  // chunks of power-of-two lengths; a length is captured the second time it
  // runs with these parameters (a serving loop changes them often)
  for (int done = 0; done < nticks;) {
    int len = 1;
    while (2 * len <= std::min(kGraphChunk, nticks - done)) len *= 2;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    for (auto &gph : b->graphs)
      if (gph.len == len) {
        exec = gph.exec;
        kernels = gph.kernels;
      }
    if (!exec && std::find(b->seen_len.begin(), b->seen_len.end(), len) == b->seen_len.end()) {
      b->seen_len.push_back(len);
      BCU(enqueue(len, &kernels));
      b->launches += kernels;
      done += len;
      continue;
    }
    if (!exec) {
      cudaGraph_t graph = nullptr;
      BCU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue(len, &kernels);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(b, FD_ECUDA, "batch graph capture: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return bfail(b, FD_ECUDA, "batch graph: %s", cudaGetErrorString(e));
      b->graphs.push_back({len, kernels, exec});
    }
    BCU(cudaGraphLaunch(exec, b->stream));
    b->launches += kernels;
    done += len;
  }
  BCU(cudaEventRecord(b->ev, b->stream));
  for (fd_ctx *c : b->members) {
    c->step += nticks;
    c->cur ^= (nticks & 1);
    if (c->nrec > 0) c->rec_rows = c->step + 1;
    if (c->stream != b->stream) BCU(cudaStreamWaitEvent(c->stream, b->ev, 0));
  }
  return FD_OK;
}

void fd_batch_destroy(fd_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->d_shots) cudaFree(b->d_shots);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_ticket) cudaFree(b->d_ticket);
  if (b->d_mem) cudaFree(b->d_mem);
  if (b->d_src) cudaFree(b->d_src);
  if (b->d_rec) cudaFree(b->d_rec);
  if (b->d_tick) cudaFree(b->d_tick);
  for (auto &gph : b->graphs) cudaGraphExecDestroy(gph.exec);
  if (b->ev) cudaEventDestroy(b->ev);
  for (int i = 0; i < 2; ++i) {
    if (b->ev_step[i]) cudaEventDestroy(b->ev_step[i]);
    if (b->ev_rec[i]) cudaEventDestroy(b->ev_rec[i]);
  }
  if (b->side) {
    cudaStreamSynchronize(b->side);
    cudaStreamDestroy(b->side);
  }
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int64_t fd_footprint_bytes(int ndim, const int64_t *shape, int space_order, int nrec, int nt,
                           int nsrc) {
  if ((ndim != 2 && ndim != 3) || !shape || space_order < 2 || space_order > 2 * kMaxR ||
      (space_order & 1) || nrec < 0 || nt < 0 || nsrc < 0)
    return -1;
  const int R = space_order / 2;
  int64_t n0 = 1, n1, n2, r0 = 0;
  if (ndim == 3) {
    n0 = shape[0]; n1 = shape[1]; n2 = shape[2]; r0 = R;
  } else {
    n1 = shape[0]; n2 = shape[1];
  }
  const int64_t px = kHaloX + (n2 + R + 31) / 32 * 32;
  const int64_t field = px * (n1 + 2 * R) * (n0 + 2 * r0) * 4;
  const int64_t npts = n0 * n1 * n2;
  const int nc = 1 << ndim;
  const int64_t rows = std::max<int64_t>(nt + 1, 1024);
  return 4 * field + 2 * npts * 4 + rows * nrec * 4 + (int64_t)nrec * nc * 12 +
         (int64_t)nsrc * nc * 24 + (int64_t)nt * nsrc * 4 + (1 << 16);
}

}  // extern "C"

// ===========================================================================
// No-allocation entry point: fd_acoustic_run_noalloc.
//
// Some callers cannot allocate GPU memory: a host application whose own pool
// (for example a framework's caching allocator) already holds the device's
// memory, or a latency-critical loop where cudaMalloc/cudaFree would stall on
// device-wide synchronisation.  This entry point runs acoustic steps on buffers
// the caller passes, keeping its working copies (the zero-halo time levels and
// the coefficient fields A and C, plus the reduction words of the set-up
// kernel) in one file-scope device array of fixed size instead of allocating.
// ===========================================================================
#include <mutex>

namespace {

constexpr size_t kNoAllocFloats = FD_NOALLOC_SCRATCH_BYTES / sizeof(float);
constexpr size_t kNoAllocStatsFloats = 64;  // 256 B for the set-up kernel's reduction words
constexpr int kNoAllocMaxDevices = 64;

// Reserved on every GPU that loads the library, until the process exits.
// Every call shares it and it keeps the last call's contents.
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

std::mutex g_noalloc_mutex;
float *g_noalloc_addr[kNoAllocMaxDevices] = {};

__global__ void k_noalloc_init_stats(unsigned *stats) {
  stats[0] = 0x7f800000u;  // identity of the min over m's bit patterns
  stats[1] = 0u;           // no invalid value seen
}

StencilFn plain_acoustic_fn(int R, bool three, bool iso2) {
#define NA_PICK(RR)                                                                    \
  case RR:                                                                             \
    return three ? k_stencil_plain<RR, kAcoustic, true>                                \
                 : (iso2 ? k_stencil_plain<RR, kAcoustic, false, true>                 \
                         : k_stencil_plain<RR, kAcoustic, false>);
  switch (R) {
    NA_PICK(1) NA_PICK(2) NA_PICK(3) NA_PICK(4) NA_PICK(5) NA_PICK(6) NA_PICK(7) NA_PICK(8)
  }
#undef NA_PICK
  return nullptr;
}

}  // namespace

#define NA_CU(call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(nullptr, FD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

extern "C" fd_status fd_acoustic_run_noalloc(int ndim, const int64_t *shape, const double *spacing,
                                             int space_order, double dt, const float *m,
                                             const float *damp, const float *u_cur,
                                             const float *u_prev, int nt, float *u_out,
                                             float *u_prev_out, void *cuda_stream) {
  g_create_error.clear();
  if (ndim != 2 && ndim != 3) return fail(nullptr, FD_EINVAL, "ndim must be 2 or 3 (got %d)", ndim);
  if (!shape || !spacing || !m || !u_cur || !u_out)
    return fail(nullptr, FD_EINVAL, "shape, spacing, m, u_cur and u_out must not be NULL");
  if (space_order < 2 || space_order > 2 * kMaxR || (space_order & 1))
    return fail(nullptr, FD_EINVAL, "space_order must be even in [2,16] (got %d)", space_order);
  if (nt < 0) return fail(nullptr, FD_EINVAL, "nt must be >= 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, FD_EINVAL, "dt must be positive and finite");
  for (int d = 0; d < ndim; ++d) {
    if (shape[d] < 2 || shape[d] > (1 << 20))
      return fail(nullptr, FD_EINVAL, "shape[%d] = %lld out of range", d, (long long)shape[d]);
    if (!(spacing[d] > 0.0) || !std::isfinite(spacing[d]))
      return fail(nullptr, FD_EINVAL, "spacing[%d] must be positive and finite", d);
  }
  // every array argument must be device memory of the current device (a host
  // address, or another GPU's memory, would be read and written from the wrong place)
  int cur_dev = 0;
  NA_CU(cudaGetDevice(&cur_dev));
  const void *ptrs[6] = {m, damp, u_cur, u_prev, u_out, u_prev_out};
  for (const void *q : ptrs) {
    if (!q) continue;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return fail(nullptr, FD_EINVAL, "array arguments must be device pointers");
    }
    if (at.type == cudaMemoryTypeDevice && at.device != cur_dev)
      return fail(nullptr, FD_EINVAL, "array argument on device %d, the current device is %d",
                  at.device, cur_dev);
  }
  const int R = space_order / 2;
  Geom g{};
  if (ndim == 3) {
    g.n0 = (int)shape[0]; g.n1 = (int)shape[1]; g.n2 = (int)shape[2];
    g.R0 = R;
  } else {
    g.n0 = 1; g.n1 = (int)shape[0]; g.n2 = (int)shape[1];
    g.R0 = 0;
  }
  g.R = R;
  g.px = kHaloX + ((g.n2 + R + 31) / 32) * 32;
  g.py = g.n1 + 2 * R;
  g.plane = (int64_t)g.px * g.py;
  g.total = g.plane * (g.n0 + 2 * g.R0);
  const size_t need = kNoAllocStatsFloats + 4 * (size_t)g.total;
  if (need > kNoAllocFloats)
    return fail(nullptr, FD_EINVAL,
                "grid needs %zu bytes of working memory (four zero-halo fields); the "
                "no-allocation entry point holds %zu bytes",
                need * sizeof(float), (size_t)FD_NOALLOC_SCRATCH_BYTES);

  // set-up, once per device: the device address of the file-scope array
  int dev = 0;
  NA_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(nullptr, FD_EUNSUPPORTED, "device %d", dev);
  float *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(nullptr, FD_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s",
                    cudaGetErrorString(e));
      g_noalloc_addr[dev] = (float *)p;
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  unsigned *stats = (unsigned *)base;
  float *lev0 = base + kNoAllocStatsFloats;
  float *lev1 = lev0 + g.total;
  float *A = lev1 + g.total;
  float *C = A + g.total;
  const int64_t n = (int64_t)g.n0 * g.n1 * g.n2;

  // the halos must start at zero; the reduction words at their identities
  NA_CU(cudaMemsetAsync(lev0, 0, 2 * g.total * sizeof(float), stream));
  k_noalloc_init_stats<<<1, 1, 0, stream>>>(stats);
  NA_CU(cudaGetLastError());
  k_scatter<<<blocks_for(n, 256), 256, 0, stream>>>(u_cur, lev0, g);
  NA_CU(cudaGetLastError());
  k_scatter<<<blocks_for(n, 256), 256, 0, stream>>>(u_prev ? u_prev : u_cur, lev1, g);
  NA_CU(cudaGetLastError());
  k_coefficients<<<blocks_for(n, 256), 256, 0, stream>>>(m, damp, A, C, g, dt, stats);
  NA_CU(cudaGetLastError());
  unsigned host_stats[2] = {0, 0};
  NA_CU(cudaMemcpyAsync(host_stats, stats, sizeof host_stats, cudaMemcpyDeviceToHost, stream));
  NA_CU(cudaStreamSynchronize(stream));
  if (host_stats[1])
    return fail(nullptr, FD_EINVAL, "m must be positive and finite, damp non-negative and finite");
  float mmin;
  std::memcpy(&mmin, &host_stats[0], sizeof mmin);
  const double S = lib_symbol(space_order);
  double lam = 0.0;
  for (int d = 0; d < ndim; ++d) lam += S / (spacing[d] * spacing[d]);
  const double dtmax = 2.0 * std::sqrt((double)mmin / lam);
  if (dt > dtmax * (1.0 + 1e-12))
    return fail(nullptr, FD_EINVAL, "dt = %g exceeds the leapfrog limit %g for min(m) = %g", dt,
                dtmax, (double)mmin);

  Coef coef;
  std::memset(&coef, 0, sizeof coef);
  double w[kMaxR + 1];
  lib_weights(space_order, w);
  for (int d = 0; d < ndim; ++d) {
    const int ax = d + 3 - ndim;
    const double s = 1.0 / (spacing[d] * spacing[d]);
    for (int k = 1; k <= R; ++k) {
      coef.w[ax][k] = (float)(w[k] * s);
      coef.wp[ax][k] = make_float2(coef.w[ax][k], coef.w[ax][k]);
    }
  }
  coef.iso2 = ndim == 2 && spacing[0] == spacing[1] ? 1 : 0;  // as fd_create sets it
  StencilFn fn = plain_acoustic_fn(R, ndim == 3, coef.iso2 != 0);
  float *cur = lev0, *prev = lev1;
  dim3 block(32, 8);
  dim3 grid((g.n2 + 31) / 32, (g.n1 + 7) / 8, g.n0);
  for (int s = 0; s < nt; ++s) {
    fn<<<grid, block, 0, stream>>>(cur, prev, A, C, g, coef);  // u^{n+1} over u^{n-1}
    NA_CU(cudaGetLastError());
    std::swap(cur, prev);
  }
  k_gather<<<blocks_for(n, 256), 256, 0, stream>>>(cur, u_out, g);
  NA_CU(cudaGetLastError());
  if (u_prev_out) {
    k_gather<<<blocks_for(n, 256), 256, 0, stream>>>(prev, u_prev_out, g);
    NA_CU(cudaGetLastError());
  }
  return FD_OK;
}
