// C ABI of the usrt library (include/usrt.h): context, resident scenes, grow-only workspaces
// charged against a memory budget, and the entry points that sequence the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/usrt.h"
#include "adjoint.cuh"
#include "bvh_build.h"
#include "image.cuh"
#include "splat.cuh"
#include "transport.cuh"

using namespace usrt;

namespace {

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

enum Slot {
  W_QA_PA, W_QA_WT, W_QA_META, W_QB_PA, W_QB_WT, W_QB_META, W_HITS, W_NEE_JOB, W_NEE_JM, W_ARR, W_CNT,
  W_ROW_CNT, W_ROW_OFF, W_ROW_CUR, W_BUCKET, W_SCRATCH, W_GTAB, W_IRF, W_ENV, W_KEY, W_PART, W_SCAL, W_GI,
  W_GRF, W_GPART, W_REC_CHUNK, W_PACK, W_NPACK, W_NEE_PATH, W_SEEDS, W_ACTIVE, W_ACT_CNT, W_RAY_KEY, W_RAY_CNT,
  W_RAY_OFF, W_RAY_CUR, W_JOBU_JOB, W_JOBU_JM, W_JOBU_PATH, W_GB, W_NEE_RES, W_NEE_XO, W_XING, W_PCLASS,
  W_ACQ_PART, W_JOB_KEY, W_JOB_CNT, W_JOB_OFF, W_JOB_CUR, W_QA_SURF, W_KEEP, W_NEE_JX, W_NEE_JW, W_JOBU_JX,
  W_JOBU_JW, W_QA_MIS, W_QB_MIS, W_SEEDV, W_DAS_ACC, W_DAS_MAX, W_COUNT
};

struct SceneGPU {
  SceneDev dev;
  float lo[3], hi[3];  // bounds of all primitives (ray-sort cells)
  std::vector<void*> allocs;
  size_t bytes = 0;
  int n_media_hint = 0;
  bool rough = false;  // theta carries a GGX roughness per medium
  int depth = 0;
};

struct StageRec {
  int stage;
  cudaEvent_t a, b;
};

struct RecordKey {
  uint64_t scene = 0, seed = 0;
  std::vector<float> theta;
  std::vector<char> acq;  // bytes of the packed Acq
  long long n_paths = 0;
  bool valid = false;
};

// A lane owns one set of workspaces, a path record and the counters of its last forward pass.
// Single-request calls run on lane 0 with the caller's stream; us_forward_batch spreads the
// requests of a batch over lanes with their own streams so that they overlap on the device.
// what the beamformed image in a lane's W_IRF workspace was made from: the RF pointer, the
// image grid and the acquisition quantities DAS reads; lets a record-mode adjoint reuse the
// forward pass's image instead of beamforming the same RF again
struct IrfKey {
  bool valid = false;
  const float* rf = nullptr;
  const void* irf = nullptr;
  std::vector<float> sig;
};

struct Lane {
  Buf ws[W_COUNT];
  Buf record;
  RecordKey rkey;
  IrfKey ikey;
  Counters* h_cnt = nullptr;  // pinned copy of the last forward's counters
  cudaEvent_t ev_stats = nullptr;
  long long last_paths = 0;
  bool stats_valid = false;
  cudaStream_t stream = nullptr;  // lane 0: none (the caller's stream)
  cudaEvent_t ev_done = nullptr;
  // second stream for the secondary rays (US_OPT_NEE_STREAM): fork events per round, a join event
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork[MAX_KMAX + 2] = {};
  cudaEvent_t ev_join = nullptr;
  cudaEvent_t ev_afork = nullptr, ev_ajoin = nullptr;  // the adjoint's fork and join
};

}  // namespace

struct us_ctx {
  int device = 0;
  size_t budget = 0, used = 0;
  std::string err;
  std::map<uint64_t, SceneGPU> scenes;
  uint64_t next_id = 1;
  std::vector<Lane*> lanes;
  Lane* L = nullptr;  // lane of the call in progress
  int num_sms = 148;
  int trav_per_sm = 4;   // blocks per SM of the traversal grid
  int march_per_sm = 4;  // resident blocks per SM of the scatterer march
  int nee_per_sm = 4;    // resident blocks per SM of the secondary-ray kernel
  int* d_status = nullptr;    // device status word of kernels outside the transport (ST_* bits)
  int opts[US_N_OPTS] = {};
  // tracing
  bool prof = false;
  std::vector<StageRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  long long launches = 0;
  long long stage_launches[US_N_STAGES] = {};
};

namespace {

int fail(us_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return fail(ctx, US_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CKS(expr)                 \
  do {                            \
    int s_ = (expr);              \
    if (s_ != US_OK) return s_;   \
  } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int dev_alloc(us_ctx* ctx, void** p, size_t bytes) {
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(ctx, US_ERR_OOM, "memory budget exceeded: %zu used + %zu requested > %zu", ctx->used, bytes,
                ctx->budget);
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, US_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->used += bytes;
  return US_OK;
}

void dev_free(us_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  ctx->used -= bytes;
}

// grow-only workspace; growing synchronises the stream before freeing the old buffer
int ws_get(us_ctx* ctx, int slot, size_t bytes, cudaStream_t st, void** out) {
  Buf& b = ctx->L->ws[slot];
  if (b.cap < bytes) {
    if (b.p) {
      CK(cudaStreamSynchronize(st));
      dev_free(ctx, b.p, b.cap);
      b.p = nullptr;
      b.cap = 0;
    }
    size_t want = bytes + bytes / 8 + 256;
    CKS(dev_alloc(ctx, &b.p, want));
    b.cap = want;
  }
  *out = b.p;
  return US_OK;
}
template <class T>
int ws(us_ctx* ctx, int slot, size_t count, cudaStream_t st, T** out) {
  void* p;
  CKS(ws_get(ctx, slot, sizeof(T) * count, st, &p));
  *out = (T*)p;
  return US_OK;
}

int grid_of(us_ctx* ctx, int per_sm) { return ctx->num_sms * per_sm; }

Lane* new_lane(us_ctx* ctx, bool own_stream) {
  Lane* l = new Lane();
  if (cudaMallocHost((void**)&l->h_cnt, sizeof(Counters)) != cudaSuccess ||
      cudaEventCreateWithFlags(&l->ev_stats, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&l->ev_done, cudaEventDisableTiming) != cudaSuccess ||
      (own_stream && cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking) != cudaSuccess)) {
    cudaGetLastError();
    delete l;
    return nullptr;
  }
  ctx->lanes.push_back(l);
  return l;
}

void free_lane(us_ctx* ctx, Lane* l) {
  for (int i = 0; i < W_COUNT; ++i)
    if (l->ws[i].p) {
      cudaFree(l->ws[i].p);
      ctx->used -= l->ws[i].cap;
    }
  if (l->record.p) {
    cudaFree(l->record.p);
    ctx->used -= l->record.cap;
  }
  if (l->h_cnt) cudaFreeHost(l->h_cnt);
  if (l->ev_stats) cudaEventDestroy(l->ev_stats);
  if (l->ev_done) cudaEventDestroy(l->ev_done);
  for (cudaEvent_t e : l->ev_fork)
    if (e) cudaEventDestroy(e);
  if (l->ev_join) cudaEventDestroy(l->ev_join);
  if (l->ev_afork) cudaEventDestroy(l->ev_afork);
  if (l->ev_ajoin) cudaEventDestroy(l->ev_ajoin);
  if (l->side) cudaStreamDestroy(l->side);
  if (l->stream) cudaStreamDestroy(l->stream);
  delete l;
}

cudaEvent_t pool_event(us_ctx* ctx) {
  if (ctx->pool_used < ctx->pool.size()) return ctx->pool[ctx->pool_used++];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  ctx->pool.push_back(e);
  ctx->pool_used++;
  return e;
}

// counts a stage's kernel launches and, while tracing, brackets them with events on the
// launching stream
struct StageScope {
  us_ctx* c;
  int stage, nk;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageScope(us_ctx* c_, int stage_, int nk_, cudaStream_t st_) : c(c_), stage(stage_), nk(nk_), st(st_) {
    if (c->prof && (a = pool_event(c))) cudaEventRecord(a, st);
  }
  ~StageScope() {
    c->launches += nk;
    c->stage_launches[stage] += nk;
    if (a) {
      cudaEvent_t b = pool_event(c);
      if (b) {
        cudaEventRecord(b, st);
        c->recs.push_back(StageRec{stage, a, b});
      }
    }
  }
};

int make_media(us_ctx* ctx, const float* theta, int M, Media& med, bool rough = false) {
  if (!theta) return fail(ctx, US_ERR_ARG, "theta is NULL");
  if (M < 1 || M > MAX_MEDIA) return fail(ctx, US_ERR_ARG, "n_media %d outside [1, %d]", M, MAX_MEDIA);
  std::memset(&med, 0, sizeof med);
  med.M = M;
  med.has_rough = rough ? 1 : 0;
  if (rough)
    for (int m = 0; m < M; ++m) {
      med.rough[m] = theta[3 * M + 2 + m];
      if (!(med.rough[m] >= 0.0f && med.rough[m] <= 1.0f))
        return fail(ctx, US_ERR_ARG, "roughness of medium %d outside [0, 1]", m);
    }
  for (int m = 0; m < M; ++m) {
    med.c[m] = theta[3 * m];
    med.rho[m] = theta[3 * m + 1];
    med.al[m] = theta[3 * m + 2];
    if (!(med.c[m] > 0) || !(med.rho[m] > 0)) return fail(ctx, US_ERR_ARG, "medium %d: c and rho must be > 0", m);
  }
  med.As = theta[3 * M];
  med.f0 = theta[3 * M + 1];
  if (!(med.f0 > 0)) return fail(ctx, US_ERR_ARG, "f0 must be > 0");
  return US_OK;
}

int make_acq(us_ctx* ctx, const us_acq_desc* d, uint64_t seed, Acq& q) {
  if (!d) return fail(ctx, US_ERR_ARG, "acq is NULL");
  std::memset(&q, 0, sizeof q);
  if (d->n_elem < 1 || d->n_elem > MAX_ELEM) return fail(ctx, US_ERR_ARG, "n_elem %d outside [1, %d]", d->n_elem, MAX_ELEM);
  if (d->n_tx < 1 || d->n_tx > MAX_TX) return fail(ctx, US_ERR_ARG, "n_tx %d outside [1, %d]", d->n_tx, MAX_TX);
  if (!d->angles) return fail(ctx, US_ERR_ARG, "angles is NULL");
  if (d->k_max < 0 || d->k_max > MAX_KMAX) return fail(ctx, US_ERR_ARG, "k_max %d outside [0, %d]", d->k_max, MAX_KMAX);
  if (d->n_samples < 4 || d->n_samples % 4 || d->n_samples > MAX_SPLAT_NS)
    return fail(ctx, US_ERR_ARG, "n_samples %d: multiple of 4 in [4, %d]", d->n_samples, MAX_SPLAT_NS);
  if (d->n_rays < 1) return fail(ctx, US_ERR_ARG, "n_rays must be >= 1");
  if (d->tx_elem >= d->n_elem) return fail(ctx, US_ERR_ARG, "tx_elem %d >= n_elem", d->tx_elem);
  if (d->tx_elem >= 0 && (d->n_tx_elem < 0 || d->tx_elem + std::max(1, d->n_tx_elem) > d->n_elem))
    return fail(ctx, US_ERR_ARG, "sub-aperture %d + %d outside the array", d->tx_elem, d->n_tx_elem);
  if (!(d->fs > 0) || !(d->pitch > 0) || !(d->c_bf > 0) || !(d->bw > 0))
    return fail(ctx, US_ERR_ARG, "fs, pitch, c_bf and bw must be > 0");
  if (d->split_mode != 0 && !(d->split_q > 0 && d->split_q < 1))
    return fail(ctx, US_ERR_ARG, "split_q must lie in (0, 1)");
  q.ne = d->n_elem;
  q.ntx = d->n_tx;
  q.ns = d->n_samples;
  q.kmax = d->k_max;
  q.nr = d->n_rays;
  q.tx_elem = d->tx_elem < 0 ? -1 : d->tx_elem;
  q.n_emit = q.tx_elem < 0 ? q.ne : std::max(1, d->n_tx_elem);
  q.split_mode = d->split_mode;
  if (d->rough_nee != 0 && d->rough_nee != 1) return fail(ctx, US_ERR_ARG, "rough_nee takes 0 or 1");
  q.rough_nee = d->rough_nee;
  q.pitch = d->pitch;
  q.hel = d->h_el;
  q.fs = d->fs;
  q.bw = d->bw;
  q.alpha_m = d->alpha_m;
  q.alpha_c = d->alpha_c;
  q.cbf = d->c_bf;
  q.split_q = d->split_q;
  q.stream = d->stream_id;
  q.key0 = (uint32_t)seed;
  q.key1 = (uint32_t)(seed >> 32);
  q.rays_per_tx = (long long)q.n_emit * q.nr;
  for (int t = 0; t < q.ntx; ++t) {
    q.sin_tx[t] = (float)std::sin((double)d->angles[t]);
    q.cos_tx[t] = (float)std::cos((double)d->angles[t]);
    q.cos_lo[t] = (float)(std::cos((double)d->angles[t]) - (double)q.cos_tx[t]);
  }
  if (q.rays_per_tx * q.ntx >= (1ll << 32) - 1) return fail(ctx, US_ERR_ARG, "too many paths (>= 2^32)");
  if ((long long)q.ntx * q.ne > 16384) return fail(ctx, US_ERR_ARG, "n_tx * n_elem > 16384");
  return US_OK;
}

int make_img(us_ctx* ctx, const us_img_desc* d, Img& im) {
  if (!d) return fail(ctx, US_ERR_ARG, "img is NULL");
  if (d->n_lines < 1) return fail(ctx, US_ERR_ARG, "n_lines must be >= 1");
  if (d->n_depth < 16 || d->n_depth > 4096 || (d->n_depth & (d->n_depth - 1)))
    return fail(ctx, US_ERR_ARG, "n_depth %d: power of two in [16, 4096]", d->n_depth);
  im.nl = d->n_lines;
  im.nd = d->n_depth;
  im.x0 = d->x0;
  im.x1 = d->x1;
  im.z0 = d->z0;
  im.z1 = d->z1;
  im.dr = d->dr_db;
  im.l1 = d->lambda1;
  im.l2 = d->lambda2;
  im.fnum = d->f_number;
  return US_OK;
}

int splat_geom(us_ctx* ctx, const Acq& q, float f0, SplatGeom& g, PulseP& P) {
  const double sig = 4.0 * std::log(2.0) / (M_PI * M_PI * (double)q.bw * q.bw * (double)f0 * f0);
  const double half = 4.0 * std::sqrt(sig) * q.fs;
  g.nrows = q.ntx * q.ne;
  g.ns = q.ns;
  g.nbins = q.ns + 2 * HALO;
  g.dlo = -(int)std::floor(half);
  const int dhi = (int)std::floor(half) + 1;
  g.ntaps = dhi - g.dlo + 1;
  g.Sig = (float)(sig * (double)q.fs * q.fs);
  g.Om = (float)(2.0 * M_PI * f0 / q.fs);
  if (g.ntaps > MAX_TAPS || dhi > HALO)
    return fail(ctx, US_ERR_ARG, "pulse support %.1f samples exceeds the splat window (%d)", half, HALO);
  P.f0 = f0;
  P.sig = (float)sig;
  P.fs = q.fs;
  P.half = (float)half;
  P.ns = q.ns;
  P.rot_c = (float)std::cos(2.0 * M_PI * (double)f0 / q.fs);
  P.rot_s = (float)std::sin(2.0 * M_PI * (double)f0 / q.fs);
  P.env_qq = (float)std::exp(-2.0 / ((double)q.fs * q.fs * sig));
  return US_OK;
}

SceneGPU* get_scene(us_ctx* ctx, uint64_t id) {
  auto it = ctx->scenes.find(id);
  if (it == ctx->scenes.end()) {
    fail(ctx, US_ERR_ARG, "unknown scene id %llu", (unsigned long long)id);
    return nullptr;
  }
  return &it->second;
}

int set_attrs(us_ctx* ctx) {
  SplatGeom g;
  g.ns = MAX_SPLAT_NS;
  g.nbins = MAX_SPLAT_NS + 2 * HALO;
  g.ntaps = MAX_TAPS;
  CK(splat_set_attrs(g));
  CK(row_scatter_set_attrs(16384));
  CK(row_hist_set_attrs(16384));
  CK(image_set_attrs(4096));
  CK(adjoint_set_attrs());
  CK(ray_sort_set_attrs());
  return US_OK;
}

struct Queues {
  PathQ a, b;
};

int alloc_queues(us_ctx* ctx, long long n, cudaStream_t st, Queues& Q) {
  CKS(ws(ctx, W_QA_PA, n, st, &Q.a.pa));
  CKS(ws(ctx, W_QA_WT, n, st, &Q.a.wt));
  CKS(ws(ctx, W_QA_META, n, st, &Q.a.meta));
  CKS(ws(ctx, W_QA_SURF, n, st, &Q.a.surf));
  Q.b.surf = nullptr;  // the sorted queue's carried hits go straight into the hit array
  Q.a.mis = Q.b.mis = nullptr;
  CKS(ws(ctx, W_QB_PA, n, st, &Q.b.pa));
  CKS(ws(ctx, W_QB_WT, n, st, &Q.b.wt));
  CKS(ws(ctx, W_QB_META, n, st, &Q.b.meta));
  return US_OK;
}

// transport of paths [path0, path0 + n): generate + (k_max + 1) rounds of traverse / interact /
// secondary rays.  arr may be null (no arrivals: decisions only).
// the lane's second stream and its events (US_OPT_NEE_STREAM), made on first use
int ensure_side(us_ctx* ctx, Lane* L) {
  if (L->side) return US_OK;
  CK(cudaStreamCreateWithFlags(&L->side, cudaStreamNonBlocking));
  for (cudaEvent_t& e : L->ev_fork) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&L->ev_join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&L->ev_afork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&L->ev_ajoin, cudaEventDisableTiming));
  return US_OK;
}

int run_transport(us_ctx* ctx, const SceneGPU* sc, const Media& med, const Acq& q, long long path0, uint32_t n,
                  Arrival* arr, uint32_t arr_cap, uint32_t* record, bool do_nee, Counters* cnt, cudaStream_t st) {
  Queues Q;
  CKS(alloc_queues(ctx, n, st, Q));
  TransportArgs A;
  std::memset(&A, 0, sizeof A);
  A.S = sc->dev;
  A.med = med;
  A.acq = q;
  CKS(ws(ctx, W_HITS, n, st, &A.hits));
  CKS(ws(ctx, W_KEEP, n, st, &A.keep));
  // secondary-ray jobs: the interaction kernel appends into `unsorted`, each round's jobs are
  // sorted into A.nee, which the secondary-ray kernel and the adjoint read
  const size_t jobs = (size_t)n * std::max(1, q.kmax);  // at most one job per path and round
  CKS(ws(ctx, W_NEE_JOB, jobs, st, &A.nee.job));
  CKS(ws(ctx, W_NEE_JM, jobs, st, &A.nee.jm));
  CKS(ws(ctx, W_NEE_PATH, jobs, st, &A.nee.jpath));
  // secondary rays start at scatterers and, with rough_nee, at rough interface events, whose
  // jobs also keep the event point and the incident direction
  const bool rough_jobs = q.rough_nee && sc->rough;
  const bool any_jobs = sc->dev.n_scat > 0 || rough_jobs;
  A.mis_on = rough_jobs;
  A.nee.jx = A.nee.jw = nullptr;
  if (rough_jobs) {
    CKS(ws(ctx, W_NEE_JX, jobs, st, &A.nee.jx));
    CKS(ws(ctx, W_NEE_JW, jobs, st, &A.nee.jw));
    CKS(ws(ctx, W_QA_MIS, n, st, &Q.a.mis));
    CKS(ws(ctx, W_QB_MIS, n, st, &Q.b.mis));
  }
  NeeQ sorted = A.nee, unsorted;
  const bool sort_jobs = any_jobs;
  if (sort_jobs) {
    CKS(ws(ctx, W_JOBU_JOB, jobs, st, &unsorted.job));
    CKS(ws(ctx, W_JOBU_JM, jobs, st, &unsorted.jm));
    CKS(ws(ctx, W_JOBU_PATH, jobs, st, &unsorted.jpath));
    unsorted.jx = unsorted.jw = nullptr;
    if (rough_jobs) {
      CKS(ws(ctx, W_JOBU_JX, jobs, st, &unsorted.jx));
      CKS(ws(ctx, W_JOBU_JW, jobs, st, &unsorted.jw));
    }
  }
  if (record && do_nee && any_jobs) {
    // secondary-ray results kept for the adjoint; crossings beyond the buffer are traced again
    CKS(ws(ctx, W_NEE_RES, jobs, st, &A.nres.res));
    CKS(ws(ctx, W_NEE_XO, jobs, st, &A.nres.xo));
    const size_t xcap = std::min<size_t>(2 * jobs, 0xFFFFFFF0u);
    CKS(ws(ctx, W_XING, xcap, st, &A.nres.xing));
    A.nres.xcap = (uint32_t)xcap;
  }
  A.arr = arr;
  A.arr_cap = arr_cap;
  A.record = record;
  A.path_base = path0;
  A.cnt = cnt;
  CK(cudaMemsetAsync(cnt, 0, sizeof(Counters), st));
  if (record) CK(cudaMemsetAsync(record, 0, sizeof(uint32_t) * (size_t)n * (q.kmax + 1), st));
  // secondary rays on the lane's second stream (US_OPT_NEE_STREAM): round k's kernel waits for
  // its sorted jobs (fork event k), and the call's stream waits for all of them at the end
  const int nee_pct = std::min(100, std::max(0, ctx->opts[US_OPT_NEE_STREAM]));
  const bool side = do_nee && any_jobs && nee_pct > 0;
  Lane* L = ctx->L;
  if (side) CKS(ensure_side(ctx, L));
  const int nee_grid = side ? std::max(ctx->num_sms, grid_of(ctx, ctx->nee_per_sm) * nee_pct / 100)
                            : grid_of(ctx, ctx->nee_per_sm);
  RaySort rs;
  for (int a = 0; a < 3; ++a) {
    const float ext = std::max(sc->hi[a] - sc->lo[a], 1e-6f);
    (&rs.lo.x)[a] = sc->lo[a];
    (&rs.inv_ext.x)[a] = 1.0f / ext;
  }
  CKS(ws(ctx, W_RAY_KEY, n, st, &rs.key));
  CKS(ws(ctx, W_RAY_CNT, RAY_BUCKETS, st, &rs.cnt));
  CKS(ws(ctx, W_RAY_OFF, RAY_BUCKETS + 1, st, &rs.off));
  A.trav_n = rs.off + RAY_KEY_BUCKETS;  // written by each round's ray sort
  CKS(ws(ctx, W_RAY_CUR, RAY_BUCKETS, st, &rs.cursor));
  // the interaction kernel keys and counts the next round's rays (A.rk) before the round's job
  // sort runs, so the job sort has scratch of its own
  A.rk = rs;
  RaySort js = rs;
  if (sort_jobs) {
    CKS(ws(ctx, W_JOB_KEY, n, st, &js.key));
    CKS(ws(ctx, W_JOB_CNT, RAY_BUCKETS, st, &js.cnt));
    CKS(ws(ctx, W_JOB_OFF, RAY_BUCKETS + 1, st, &js.off));
    CKS(ws(ctx, W_JOB_CUR, RAY_BUCKETS, st, &js.cursor));
  }
  // Q.a: rays as the interaction kernel appends them; Q.b: coherence-sorted (the emission
  // writes there directly)
  A.qout = Q.b;
  {
    StageScope sc_(ctx, US_STAGE_GENERATE, 3, st);
    CK(cudaMemsetAsync(rs.cnt, 0, sizeof(uint32_t) * RAY_BUCKETS, st));
    launch_generate(A, path0, n, rs, grid_of(ctx, 2), st);
  }
  for (int k = 0; k <= q.kmax; ++k) {
    A.k = k;
    if (k > 0) {
      StageScope sc_(ctx, US_STAGE_RAY_SORT, 2, st);
      launch_ray_sort(A, Q.a, Q.b, rs, grid_of(ctx, 2), st);
    }
    A.qin = Q.b;
    A.qout = Q.a;
    if (sort_jobs) A.nee = unsorted;
    {
      StageScope sc_(ctx, US_STAGE_TRAVERSE, sc->dev.n_scat > 0 ? 2 : 1, st);
      launch_traverse(A, grid_of(ctx, ctx->trav_per_sm), st);
      if (sc->dev.n_scat > 0) launch_march(A, grid_of(ctx, ctx->march_per_sm), st);
    }
    {
      StageScope sc_(ctx, US_STAGE_INTERACT, 1, st);
      CK(cudaMemsetAsync(rs.cnt, 0, sizeof(uint32_t) * RAY_BUCKETS, st));  // this round's sort has scanned them
      launch_interact(A, grid_of(ctx, 8), st);
    }
    // the round's secondary rays (job sort, then the kernel): on the second stream from here
    cudaStream_t ns = st;
    if (side) {
      CK(cudaEventRecord(L->ev_fork[k], st));
      CK(cudaStreamWaitEvent(L->side, L->ev_fork[k], 0));
      ns = L->side;
    }
    if (sort_jobs && k < q.kmax) {
      StageScope sc_(ctx, US_STAGE_JOB_SORT, 3, ns);
      launch_job_sort(A, unsorted, sorted, js, grid_of(ctx, 2), ns);
    }
    A.nee = sorted;
    if (do_nee && any_jobs) {
      StageScope sc_(ctx, US_STAGE_NEE, 1, ns);
      launch_nee(A, nee_grid, ns);
    }
  }
  if (side) {
    CK(cudaEventRecord(L->ev_join, L->side));
    CK(cudaStreamWaitEvent(st, L->ev_join, 0));
  }
  CK(cudaGetLastError());
  return US_OK;
}

int do_splat(us_ctx* ctx, const Acq& q, float f0, const Arrival* arr, const uint32_t* n_arr, uint32_t cap, float* rf,
             cudaStream_t st) {
  SplatGeom g;
  PulseP P;
  CKS(splat_geom(ctx, q, f0, g, P));
  SplatWork w;
  CKS(ws(ctx, W_ROW_CNT, g.nrows, st, &w.row_cnt));
  CKS(ws(ctx, W_ROW_OFF, g.nrows + 1, st, &w.row_off));
  CKS(ws(ctx, W_ROW_CUR, g.nrows, st, &w.row_cursor));
  CKS(ws(ctx, W_BUCKET, (size_t)cap + 1, st, &w.bucket));
  CKS(ws(ctx, W_SCRATCH, (size_t)cap + 1, st, &w.scratch));
  float* G;
  CKS(ws(ctx, W_GTAB, K_MOM * MAX_TAPS, st, &G));
  {
    StageScope sc_(ctx, US_STAGE_SPLAT_SORT, 4, st);
    launch_pulse_table(g, G, st);
    launch_splat_sort(g, arr, n_arr, cap, w, grid_of(ctx, 4), st);
  }
  {
    StageScope sc_(ctx, US_STAGE_SPLAT_ROWS, 1, st);
    launch_splat_rows(g, w, G, rf, st);
  }
  CK(cudaGetLastError());
  return US_OK;
}

std::vector<float> das_signature(const Acq& q, const Img& im) {
  std::vector<float> v = {(float)q.ne, q.pitch, (float)q.ntx, q.fs, (float)q.ns, q.cbf, (float)im.nl, (float)im.nd,
                          im.x0, im.x1, im.z0, im.z1, im.fnum};
  for (int t = 0; t < q.ntx; ++t) {
    v.push_back(q.sin_tx[t]);
    v.push_back(q.cos_tx[t]);
    v.push_back(q.cos_lo[t]);
  }
  return v;
}

void irf_made(us_ctx* ctx, const Acq& q, const Img& im, const float* rf, const float* irf) {
  IrfKey& k = ctx->L->ikey;
  k.valid = true;
  k.rf = rf;
  k.irf = irf;
  k.sig = das_signature(q, im);
}

int do_bmode(us_ctx* ctx, const Acq& q, const Img& im, const float* rf, float* bmode, cudaStream_t st) {
  float *irf, *env;
  unsigned long long* key;
  CKS(ws(ctx, W_IRF, (size_t)im.nl * im.nd, st, &irf));
  CKS(ws(ctx, W_ENV, (size_t)im.nl * im.nd, st, &env));
  CKS(ws(ctx, W_KEY, 2, st, &key));
  {
    StageScope sc_(ctx, US_STAGE_DAS, 1, st);
    launch_das(q, im, rf, irf, grid_of(ctx, 8), st, ctx->opts[US_OPT_DAS_TMA] ? ctx->d_status : nullptr);
  }
  irf_made(ctx, q, im, rf, irf);
  {
    StageScope sc_(ctx, US_STAGE_ENVLOG, 0, st);
    sc_.nk = launch_envlog(im, irf, env, key, bmode, grid_of(ctx, 8), st, ctx->d_status,
                           ctx->opts[US_OPT_FAULT_BARRIER]);
  }
  CK(cudaGetLastError());
  return US_OK;
}

}  // namespace

// =========================================================================================
namespace usrt {  // optim.cu
void launch_param_map(int n, const float* theta_u, const float* lo, const float* hi, float* theta, cudaStream_t st);
void launch_adam_step(int n, float* theta_u, const float* grad, const float* lo, const float* hi, const float* lr,
                      float beta1, float beta2, float eps, float clip_norm, float bc1, float bc2, float* m, float* v,
                      cudaStream_t st);
}  // namespace usrt

extern "C" {

int us_create(us_ctx** out, int device, size_t mem_budget_bytes) {
  if (!out) return US_ERR_ARG;
  *out = nullptr;
  us_ctx* ctx = new us_ctx();
  ctx->device = device;
  ctx->budget = mem_budget_bytes;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return US_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  ctx->L = new_lane(ctx, false);
  if (!ctx->L) {
    delete ctx;
    return US_ERR_CUDA;
  }
  ctx->opts[US_OPT_LANES] = 4;
  ctx->opts[US_OPT_NEE_STREAM] = 100;
  ctx->trav_per_sm = traverse_blocks_per_sm();
  ctx->march_per_sm = march_blocks_per_sm();
  ctx->nee_per_sm = nee_blocks_per_sm();
  if (dev_alloc(ctx, (void**)&ctx->d_status, 256) != US_OK || cudaMemset(ctx->d_status, 0, 256) != cudaSuccess) {
    delete ctx;
    return US_ERR_OOM;
  }
  if (set_attrs(ctx) != US_OK) {
    delete ctx;
    return US_ERR_CUDA;
  }
  *out = ctx;
  return US_OK;
}

void us_destroy(us_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->scenes)
    for (void* p : kv.second.allocs) cudaFree(p);
  for (Lane* l : ctx->lanes) free_lane(ctx, l);
  ctx->lanes.clear();
  ctx->L = nullptr;
  if (ctx->d_status) cudaFree(ctx->d_status);
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
}

int us_profile(us_ctx* ctx, int enable) {
  if (!ctx) return US_ERR_ARG;
  ctx->prof = enable != 0;
  ctx->recs.clear();
  ctx->pool_used = 0;
  for (int i = 0; i < US_N_STAGES; ++i) ctx->stage_launches[i] = 0;
  return US_OK;
}

int us_profile_read(us_ctx* ctx, double* ms, int64_t* launches, int n) {
  if (!ctx || n < 0 || (n && (!ms || !launches))) return fail(ctx, US_ERR_ARG, "invalid arguments");
  std::vector<double> acc(US_N_STAGES, 0.0);
  for (const StageRec& r : ctx->recs) {
    CK(cudaEventSynchronize(r.b));
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    acc[r.stage] += t;
  }
  for (int i = 0; i < n && i < US_N_STAGES; ++i) {
    ms[i] = acc[i];
    launches[i] = ctx->stage_launches[i];
  }
  ctx->recs.clear();
  ctx->pool_used = 0;
  for (int i = 0; i < US_N_STAGES; ++i) ctx->stage_launches[i] = 0;
  return US_OK;
}

int us_param_map(us_ctx* ctx, int n, const float* theta_u_dev, const float* lo_dev, const float* hi_dev,
                 float* theta_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  if (n < 1 || n > 1024 || !theta_u_dev || !lo_dev || !hi_dev || !theta_dev)
    return fail(ctx, US_ERR_ARG, "param_map: 1 <= n <= 1024 and four device arrays");
  CK(cudaSetDevice(ctx->device));
  StageScope sc_(ctx, US_STAGE_OTHER, 1, (cudaStream_t)stream);
  launch_param_map(n, theta_u_dev, lo_dev, hi_dev, theta_dev, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return US_OK;
}

int us_adam_step(us_ctx* ctx, int n, float* theta_u_dev, const float* dL_dtheta_dev, const float* lo_dev,
                 const float* hi_dev, const float* lr_dev, float beta1, float beta2, float eps, float clip_norm,
                 int step, float* m_dev, float* v_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  if (n < 1 || n > 1024 || !theta_u_dev || !dL_dtheta_dev || !lo_dev || !hi_dev || !lr_dev || !m_dev || !v_dev)
    return fail(ctx, US_ERR_ARG, "adam_step: 1 <= n <= 1024 and seven device arrays");
  if (step < 1 || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return fail(ctx, US_ERR_ARG, "adam_step: step >= 1, 0 <= beta < 1, eps > 0");
  CK(cudaSetDevice(ctx->device));
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
  StageScope sc_(ctx, US_STAGE_OTHER, 1, (cudaStream_t)stream);
  launch_adam_step(n, theta_u_dev, dL_dtheta_dev, lo_dev, hi_dev, lr_dev, beta1, beta2, eps, clip_norm, bc1, bc2,
                   m_dev, v_dev, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return US_OK;
}

int us_set_option(us_ctx* ctx, int option, int value) {
  if (!ctx || option < 0 || option >= US_N_OPTS) return fail(ctx, US_ERR_ARG, "unknown option %d", option);
  if (option == US_OPT_FAULT_BARRIER && value != 0 && value != 1)
    return fail(ctx, US_ERR_ARG, "US_OPT_FAULT_BARRIER takes 0 or 1");
  ctx->opts[option] = value;
  return US_OK;
}

int us_get_status(us_ctx* ctx, int clear, int* device_status) {
  if (!ctx || !device_status) return fail(ctx, US_ERR_ARG, "null argument");
  CK(cudaSetDevice(ctx->device));
  CK(cudaDeviceSynchronize());
  int ds = 0;
  CK(cudaMemcpy(&ds, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (clear) CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
  *device_status = (ds & ST_OVERFLOW) ? US_ERR_OVERFLOW : ((ds & ST_TIMEOUT) ? US_ERR_TIMEOUT : US_OK);
  return US_OK;
}

int us_launch_count(us_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return US_ERR_ARG;
  *n = ctx->launches;
  return US_OK;
}

const char* us_last_error(us_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int us_memory(us_ctx* ctx, size_t* used, size_t* budget) {
  if (!ctx) return US_ERR_ARG;
  if (used) *used = ctx->used;
  if (budget) *budget = ctx->budget;
  return US_OK;
}

int us_scene_upload(us_ctx* ctx, const us_scene_desc* d, uint64_t* scene_id) {
  if (!ctx || !d || !scene_id) return fail(ctx, US_ERR_ARG, "null argument");
  if (d->n_tris < 0 || d->n_scat < 0 || (d->n_tris && (!d->tris || !d->media)) ||
      (d->n_scat && (!d->scat_pos || !d->scat_amp)))
    return fail(ctx, US_ERR_ARG, "invalid scene arrays");
  if (d->n_tris >= (1 << 20) || d->n_scat >= (1 << 20))
    return fail(ctx, US_ERR_ARG, "at most 2^20 - 1 triangles and scatterers");
  if (d->n_media < 1 || d->n_media > MAX_MEDIA) return fail(ctx, US_ERR_ARG, "n_media outside [1, %d]", MAX_MEDIA);
  for (int i = 0; i < 2 * d->n_tris; ++i)
    if (d->media[i] < 0 || d->media[i] >= d->n_media) return fail(ctx, US_ERR_ARG, "triangle medium out of range");
  CK(cudaSetDevice(ctx->device));
  HostSceneIn in;
  in.n_tris = d->n_tris;
  in.tris = d->tris;
  in.media = d->media;
  in.n_scat = d->n_scat;
  in.scat_pos = d->scat_pos;
  in.scat_amp = d->scat_amp;
  in.r_s = d->r_s;
  HostSceneOut o;
  build_scene_host(in, o);
  if (o.gn[0] < 0) return fail(ctx, US_ERR_ARG, "more than 255 scatterer spheres overlap one grid cell at every cell size");
  SceneGPU sc;
  sc.n_media_hint = d->n_media;
  sc.rough = d->rough != 0;
  auto up_bytes = [&](const void* src, size_t bytes, const void** dst) -> int {
    void* p = nullptr;
    CKS(dev_alloc(ctx, &p, bytes));
    sc.allocs.push_back(p);
    sc.bytes += bytes;
    if (bytes) CK(cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice));
    *dst = p;
    return US_OK;
  };
  auto up = [&](const std::vector<float>& v, const float4** dst) -> int {
    return up_bytes(v.data(), v.size() * sizeof(float), reinterpret_cast<const void**>(dst));
  };
  int s;
  if ((s = up(o.tri_nrm, &sc.dev.tri_nrm)) || (s = up(o.tri_v0, &sc.dev.tri_v0)) || (s = up(o.tri_e1, &sc.dev.tri_e1)) ||
      (s = up(o.tri_e2, &sc.dev.tri_e2)) || (s = up(o.scat, &sc.dev.scat)) ||
      (s = up(o.nodes_t, &sc.dev.nodes_t)) || (s = up(o.prims_t, &sc.dev.prims_t)) ||
      (s = up(o.nodes4, &sc.dev.nodes4)) ||
      (s = up(o.cell_sph, &sc.dev.cell_sph)) || (s = up(o.cell2, &sc.dev.cell2)) ||
      (s = up_bytes(o.cell.data(), o.cell.size() * sizeof(uint32_t), reinterpret_cast<const void**>(&sc.dev.cell)))) {
    for (void* p : sc.allocs) cudaFree(p);
    ctx->used -= sc.bytes;
    return s;
  }
  // scene bounds (ray-sort cells): the triangle BVH's root box (union of node 0's two child
  // boxes: x at words (0,1)/(4,5), y at (2,3)/(6,7), z at (8,9)/(10,11)) and the scatterer grid
  const int lo_w[3][2] = {{0, 4}, {2, 6}, {8, 10}};
  const float glo[3] = {o.glo[0], o.glo[1], o.glo[2]};
  for (int a = 0; a < 3; ++a) {
    sc.lo[a] = 3.0e38f;
    sc.hi[a] = -3.0e38f;
    if (d->n_tris) {
      sc.lo[a] = std::min(o.nodes_t[lo_w[a][0]], o.nodes_t[lo_w[a][1]]);
      sc.hi[a] = std::max(o.nodes_t[lo_w[a][0] + 1], o.nodes_t[lo_w[a][1] + 1]);
    }
    if (d->n_scat) {
      sc.lo[a] = std::min(sc.lo[a], glo[a]);
      sc.hi[a] = std::max(sc.hi[a], glo[a] + o.gn[a] * o.gh);
    }
    if (!(sc.lo[a] <= sc.hi[a])) {
      sc.lo[a] = -1.0f;
      sc.hi[a] = 1.0f;
    }
  }
  sc.dev.glo = make_float3(o.glo[0], o.glo[1], o.glo[2]);
  sc.dev.gh = o.gh;
  sc.dev.gnx = o.gn[0];
  sc.dev.gny = o.gn[1];
  sc.dev.gnz = o.gn[2];
  sc.dev.n_tris = d->n_tris;
  sc.dev.n_scat = d->n_scat;
  sc.dev.rs2 = d->r_s * d->r_s;
  // depth check: the traversal stacks hold 64 entries
  sc.depth = std::max(o.depth_t, 3 * o.depth4 + 1);  // a 4-wide node pushes up to 3 entries
  if (sc.depth > 60) {
    for (void* p : sc.allocs) cudaFree(p);
    ctx->used -= sc.bytes;
    return fail(ctx, US_ERR_ARG, "BVH depth %d exceeds the traversal stack", sc.depth);
  }
  uint64_t id = ctx->next_id++;
  ctx->scenes[id] = sc;
  *scene_id = id;
  return US_OK;
}

int us_scene_release(us_ctx* ctx, uint64_t scene_id) {
  if (!ctx) return US_ERR_ARG;
  SceneGPU* sc = get_scene(ctx, scene_id);
  if (!sc) return US_ERR_ARG;
  CK(cudaDeviceSynchronize());
  for (void* p : sc->allocs) cudaFree(p);
  ctx->used -= sc->bytes;
  ctx->scenes.erase(scene_id);
  for (Lane* l : ctx->lanes)
    if (l->rkey.scene == scene_id) l->rkey.valid = false;
  return US_OK;
}

int us_philox_fill(us_ctx* ctx, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                   int64_t n, uint32_t* out_dev, void* stream) {
  if (!ctx || (n > 0 && !out_dev) || n < 0) return fail(ctx, US_ERR_ARG, "invalid arguments");
  if (!aligned16(out_dev)) return fail(ctx, US_ERR_ARG, "out_dev must be 16-byte aligned");
  if (n == 0) return US_OK;
  StageScope sc_(ctx, US_STAGE_OTHER, 1, (cudaStream_t)stream);
  launch_philox_fill(c0, c1, c2, c3, k0, k1, n, out_dev, grid_of(ctx, 8), (cudaStream_t)stream);
  CK(cudaGetLastError());
  return US_OK;
}

int us_forward(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, const us_img_desc* img,
               uint64_t seed, int keep_record, float* rf_dev, float* bmode_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SceneGPU* sc = get_scene(ctx, scene);
  if (!sc) return US_ERR_ARG;
  if (!rf_dev || !aligned16(rf_dev) || (bmode_dev && !aligned16(bmode_dev)))
    return fail(ctx, US_ERR_ARG, "rf_dev / bmode_dev must be non-null (rf) and 16-byte aligned");
  Media med;
  Acq q;
  Img im;
  CKS(make_media(ctx, theta, sc->n_media_hint, med, sc->rough));
  CKS(make_acq(ctx, acq, seed, q));
  if (bmode_dev) CKS(make_img(ctx, img, im));
  ctx->L->rkey.valid = false;  // job buffers and counters are about to be overwritten
  ctx->L->ikey.valid = false;  // and rf_dev, which the lane's beamformed image may have come from
  const long long n_paths = q.rays_per_tx * q.ntx;
  const long long cap_ll = n_paths * (q.kmax + 1);
  const uint32_t cap = (uint32_t)std::min<long long>(cap_ll, 0xFFFFFFF0ll);
  Arrival* arr;
  Counters* cnt;
  CKS(ws(ctx, W_ARR, cap, st, &arr));
  CKS(ws(ctx, W_CNT, 1, st, &cnt));
  uint32_t* record = nullptr;
  if (keep_record) {
    size_t bytes = sizeof(uint32_t) * (size_t)n_paths * (q.kmax + 1);
    if (ctx->L->record.cap < bytes) {
      if (ctx->L->record.p) {
        CK(cudaStreamSynchronize(st));
        dev_free(ctx, ctx->L->record.p, ctx->L->record.cap);
        ctx->L->record.p = nullptr;
        ctx->L->record.cap = 0;
      }
      CKS(dev_alloc(ctx, &ctx->L->record.p, bytes));
      ctx->L->record.cap = bytes;
    }
    record = (uint32_t*)ctx->L->record.p;
  }
  CKS(run_transport(ctx, sc, med, q, 0, (uint32_t)n_paths, arr, cap, record, true, cnt, st));
  CKS(do_splat(ctx, q, med.f0, arr, &cnt->n_arr, cap, rf_dev, st));
  if (bmode_dev) CKS(do_bmode(ctx, q, im, rf_dev, bmode_dev, st));
  CK(cudaMemcpyAsync(ctx->L->h_cnt, cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(ctx->L->ev_stats, st));
  ctx->L->last_paths = n_paths;
  ctx->L->stats_valid = true;
  if (keep_record) {
    ctx->L->rkey.scene = scene;
    ctx->L->rkey.seed = seed;
    ctx->L->rkey.theta.assign(theta, theta + n_theta(med));
    ctx->L->rkey.acq.assign((const char*)&q, (const char*)&q + sizeof q);
    ctx->L->rkey.n_paths = n_paths;
    ctx->L->rkey.valid = true;
  }
  return US_OK;
}

int us_get_stats(us_ctx* ctx, us_stats* out) {
  if (!ctx || !out) return US_ERR_ARG;
  if (!ctx->L->stats_valid) return fail(ctx, US_ERR_STATE, "no forward pass yet");
  CK(cudaEventSynchronize(ctx->L->ev_stats));
  const Counters& c = *ctx->L->h_cnt;
  out->n_paths = ctx->L->last_paths;
  long long seg = 0, nee = 0;
  for (int k = 0; k <= MAX_KMAX; ++k) {
    seg += c.live[k];
    nee += c.nee[k];
  }
  out->segments = seg;
  out->nee_queries = nee;
  static_assert(US_MAX_ROUNDS == MAX_KMAX + 2, "rounds");
  for (int k = 0; k < US_MAX_ROUNDS; ++k) out->live[k] = k <= MAX_KMAX ? c.live[k] : 0;
  out->pad = 0;
  out->arrivals = c.n_arr;
  out->dropped = c.dropped;
  int ds = 0;
  CK(cudaMemcpy(&ds, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  const int st_bits = c.status | ds;
  out->status = (st_bits & ST_OVERFLOW) ? US_ERR_OVERFLOW : (st_bits & ST_TIMEOUT ? US_ERR_TIMEOUT : 0);
  return US_OK;
}

int us_get_record(us_ctx* ctx, int64_t path_lo, int64_t n, uint32_t* out_dev, void* stream) {
  if (!ctx || !out_dev || n < 0 || path_lo < 0) return fail(ctx, US_ERR_ARG, "invalid arguments");
  if (!ctx->L->rkey.valid) return fail(ctx, US_ERR_STATE, "no record kept");
  if (path_lo + n > ctx->L->rkey.n_paths) return fail(ctx, US_ERR_ARG, "path range outside the record");
  const Acq* q = (const Acq*)ctx->L->rkey.acq.data();
  const size_t K1 = q->kmax + 1;
  CK(cudaMemcpyAsync(out_dev, (uint32_t*)ctx->L->record.p + (size_t)path_lo * K1, sizeof(uint32_t) * (size_t)n * K1,
                     cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return US_OK;
}

int us_get_arrivals(us_ctx* ctx, int64_t lo, int64_t n, uint32_t* out_dev, void* stream) {
  if (!ctx || (n && !out_dev) || n < 0 || lo < 0) return fail(ctx, US_ERR_ARG, "invalid arguments");
  if (!ctx->L->stats_valid) return fail(ctx, US_ERR_STATE, "no forward pass yet");
  CK(cudaEventSynchronize(ctx->L->ev_stats));
  // the list of the lane's last forward pass: only us_forward writes (or grows) W_ARR
  const Buf& b = ctx->L->ws[W_ARR];
  const long long have = std::min<long long>(ctx->L->h_cnt->n_arr, (long long)(b.cap / sizeof(Arrival)));
  if (lo + n > have) return fail(ctx, US_ERR_ARG, "arrival range outside the list");
  if (!n) return US_OK;
  CK(cudaMemcpyAsync(out_dev, (const Arrival*)b.p + lo, sizeof(Arrival) * (size_t)n, cudaMemcpyDeviceToDevice,
                     (cudaStream_t)stream));
  return US_OK;
}

int us_splat(us_ctx* ctx, const us_acq_desc* acq, float f0, int64_t n, const int32_t* tx_dev, const int32_t* e_dev,
             const float* tau_dev, const float* a_dev, float* rf_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Acq q;
  CKS(make_acq(ctx, acq, 0, q));
  if (n < 0 || n >= 0xFFFFFFF0ll || !rf_dev || !aligned16(rf_dev) || (n && (!tx_dev || !e_dev || !tau_dev || !a_dev)))
    return fail(ctx, US_ERR_ARG, "invalid arrival list");
  ctx->L->ikey.valid = false;  // rf_dev is rewritten
  Arrival* arr;
  uint32_t* n_out;
  CKS(ws(ctx, W_PACK, (size_t)n + 1, st, &arr));
  CKS(ws(ctx, W_NPACK, 1, st, &n_out));
  CK(cudaMemsetAsync(n_out, 0, sizeof(uint32_t), st));
  if (n) {
    StageScope sc_(ctx, US_STAGE_OTHER, 1, st);
    launch_pack_arrivals(tx_dev, e_dev, tau_dev, a_dev, n, q.ne, q.fs, arr, n_out, grid_of(ctx, 4), st);
  }
  return do_splat(ctx, q, f0, arr, n_out, (uint32_t)n + 1, rf_dev, st);
}

int us_das(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev, float* irf_dev,
           void* stream) {
  if (!ctx) return US_ERR_ARG;
  Acq q;
  Img im;
  CKS(make_acq(ctx, acq, 0, q));
  CKS(make_img(ctx, img, im));
  if (!rf_dev || !irf_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  StageScope sc_(ctx, US_STAGE_DAS, 1, (cudaStream_t)stream);
  launch_das(q, im, rf_dev, irf_dev, grid_of(ctx, 8), (cudaStream_t)stream,
             ctx->opts[US_OPT_DAS_TMA] ? ctx->d_status : nullptr);
  CK(cudaGetLastError());
  return US_OK;
}

int us_envlog(us_ctx* ctx, const us_img_desc* img, const float* irf_dev, float* bmode_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Img im;
  CKS(make_img(ctx, img, im));
  if (!irf_dev || !bmode_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  float* env;
  unsigned long long* key;
  CKS(ws(ctx, W_ENV, (size_t)im.nl * im.nd, st, &env));
  CKS(ws(ctx, W_KEY, 2, st, &key));
  StageScope sc_(ctx, US_STAGE_ENVLOG, 0, st);
  sc_.nk = launch_envlog(im, irf_dev, env, key, bmode_dev, grid_of(ctx, 8), st, ctx->d_status,
                         ctx->opts[US_OPT_FAULT_BARRIER]);
  CK(cudaGetLastError());
  return US_OK;
}

int us_bmode(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev, float* bmode_dev,
             void* stream) {
  if (!ctx) return US_ERR_ARG;
  Acq q;
  Img im;
  CKS(make_acq(ctx, acq, 0, q));
  CKS(make_img(ctx, img, im));
  if (!rf_dev || !bmode_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  return do_bmode(ctx, q, im, rf_dev, bmode_dev, (cudaStream_t)stream);
}

int us_loss(us_ctx* ctx, const us_img_desc* img, const float* bmode_dev, const float* bref_dev, float* loss_dev,
            float* dL_dB_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Img im;
  CKS(make_img(ctx, img, im));
  if (!bmode_dev || !bref_dev || !loss_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  float* part;
  const int np = grid_of(ctx, 2);
  CKS(ws(ctx, W_PART, np, st, &part));
  StageScope sc_(ctx, US_STAGE_LOSS, 2, st);
  launch_loss(im, bmode_dev, bref_dev, dL_dB_dev, part, np, loss_dev, st);
  CK(cudaGetLastError());
  return US_OK;
}

int us_envlog_vjp(us_ctx* ctx, const us_img_desc* img, const float* irf_dev, const float* dL_dB_dev,
                  float* dL_dirf_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Img im;
  CKS(make_img(ctx, img, im));
  if (!irf_dev || !dL_dB_dev || !dL_dirf_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  float *env, *part, *scal;
  unsigned long long* key;
  const int np = grid_of(ctx, 2);
  CKS(ws(ctx, W_ENV, (size_t)im.nl * im.nd, st, &env));
  CKS(ws(ctx, W_KEY, 2, st, &key));
  CKS(ws(ctx, W_PART, np, st, &part));
  CKS(ws(ctx, W_SCAL, 4, st, &scal));
  StageScope sc_(ctx, US_STAGE_ENVLOG_VJP, 4, st);
  launch_envlog_vjp(im, irf_dev, dL_dB_dev, env, key, part, np, scal, dL_dirf_dev, grid_of(ctx, 8), st);
  CK(cudaGetLastError());
  return US_OK;
}

int us_das_adjoint(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* dL_dirf_dev,
                   float* dL_drf_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  Acq q;
  Img im;
  CKS(make_acq(ctx, acq, 0, q));
  CKS(make_img(ctx, img, im));
  if (!dL_dirf_dev || !dL_drf_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  unsigned long long* acc;
  unsigned int* maxbits;
  CKS(ws(ctx, W_DAS_ACC, (size_t)q.ntx * q.ne * q.ns, (cudaStream_t)stream, &acc));
  CKS(ws(ctx, W_DAS_MAX, 1, (cudaStream_t)stream, &maxbits));
  StageScope sc_(ctx, US_STAGE_DAS_ADJ, 3, (cudaStream_t)stream);
  launch_das_adj(q, im, dL_dirf_dev, dL_drf_dev, grid_of(ctx, 8), (cudaStream_t)stream, acc, maxbits);
  CK(cudaGetLastError());
  return US_OK;
}

// reuse_irf: the lane's beamformed image may be reused when it was made from rf_dev with the
// same grid and acquisition (a record-mode adjoint right after its forward pass)
static int bmode_vjp(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev,
                     const float* dL_dB_dev, float* dL_drf_dev, void* stream, bool reuse_irf) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Acq q;
  Img im;
  CKS(make_acq(ctx, acq, 0, q));
  CKS(make_img(ctx, img, im));
  if (!rf_dev || !dL_dB_dev || !dL_drf_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  float *irf, *gi;
  CKS(ws(ctx, W_IRF, (size_t)im.nl * im.nd, st, &irf));
  CKS(ws(ctx, W_GI, (size_t)im.nl * im.nd, st, &gi));
  const IrfKey& k = ctx->L->ikey;
  if (!(reuse_irf && k.valid && k.rf == rf_dev && k.irf == irf && k.sig == das_signature(q, im))) {
    StageScope sc_(ctx, US_STAGE_DAS, 1, st);
    launch_das(q, im, rf_dev, irf, grid_of(ctx, 8), st, ctx->opts[US_OPT_DAS_TMA] ? ctx->d_status : nullptr);
    irf_made(ctx, q, im, rf_dev, irf);
  }
  unsigned long long* acc;
  unsigned int* maxbits;
  CKS(ws(ctx, W_DAS_ACC, (size_t)q.ntx * q.ne * q.ns, st, &acc));
  CKS(ws(ctx, W_DAS_MAX, 1, st, &maxbits));
  CKS(us_envlog_vjp(ctx, img, irf, dL_dB_dev, gi, stream));
  {
    StageScope sc_(ctx, US_STAGE_DAS_ADJ, 3, st);
    launch_das_adj(q, im, gi, dL_drf_dev, grid_of(ctx, 8), st, acc, maxbits);
  }
  CK(cudaGetLastError());
  return US_OK;
}

int us_bmode_vjp(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev,
                 const float* dL_dB_dev, float* dL_drf_dev, void* stream) {
  return bmode_vjp(ctx, acq, img, rf_dev, dL_dB_dev, dL_drf_dev, stream, false);
}

int us_splat_adjoint(us_ctx* ctx, const us_acq_desc* acq, float f0, int64_t n, const int32_t* tx_dev,
                     const int32_t* e_dev, const float* tau_dev, const float* a_dev, const float* dL_drf_dev,
                     float* ga_dev, float* gt_dev, float* gf_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  Acq q;
  CKS(make_acq(ctx, acq, 0, q));
  SplatGeom g;
  PulseP P;
  CKS(splat_geom(ctx, q, f0, g, P));
  if (n < 0 || (n && (!tx_dev || !e_dev || !tau_dev || !a_dev || !dL_drf_dev || !ga_dev || !gt_dev || !gf_dev)))
    return fail(ctx, US_ERR_ARG, "invalid arrival list");
  if (n) {
    StageScope sc_(ctx, US_STAGE_OTHER, 1, (cudaStream_t)stream);
    launch_splat_adjoint(q, P, tx_dev, e_dev, tau_dev, a_dev, n, dL_drf_dev, ga_dev, gt_dev, gf_dev, grid_of(ctx, 4),
                         (cudaStream_t)stream);
  }
  CK(cudaGetLastError());
  return US_OK;
}

// dL_dacq_dev != NULL: also the acquisition gradient (c_bf, pitch, steering angles) through the
// emission and the secondary rays' targets, written (or added when acc_acq) to
// dL_dacq_dev[2 + ntx]
// dL_dtris_dev != NULL: also dL/d(triangle vertices) [n_tris][9] (overwritten)
static int transport_vjp(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, uint64_t seed,
                         int mode, const float* dL_drf_dev, float* dL_dtheta_dev, float* dL_dacq_dev, int acc_acq,
                         void* stream, float* dL_dtris_dev = nullptr) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SceneGPU* sc = get_scene(ctx, scene);
  if (!sc) return US_ERR_ARG;
  if (!dL_drf_dev || !dL_dtheta_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  Media med;
  Acq q;
  CKS(make_media(ctx, theta, sc->n_media_hint, med, sc->rough));
  CKS(make_acq(ctx, acq, seed, q));
  SplatGeom g;
  AdjArgs A;
  std::memset(&A, 0, sizeof A);
  CKS(splat_geom(ctx, q, med.f0, g, A.pulse));
  A.S = sc->dev;
  A.med = med;
  A.acq = q;
  A.grf = dL_drf_dev;
  const int Ps = n_theta(med);
  A.P = Ps;
  A.acq_slot = -1;
  if (dL_dacq_dev) {
    A.acq_slot = Ps;
    A.P = Ps + 2 + q.ntx;
  }
  A.g_tris = dL_dtris_dev;
  if (dL_dtris_dev && sc->dev.n_tris)
    CK(cudaMemsetAsync(dL_dtris_dev, 0, sizeof(float) * 9 * (size_t)sc->dev.n_tris, st));
  const int grid = grid_of(ctx, 8);
  float* gpart;  // [0, grid) rows: path sweep; [grid, 2 grid): secondary rays
  CKS(ws(ctx, W_GPART, (size_t)2 * grid * A.P, st, &gpart));
  const long long n_paths = q.rays_per_tx * q.ntx;
  const int K1 = q.kmax + 1;
  uint32_t *work, *active;
  const auto sweep = [&](const uint32_t* rec, long long p0, uint32_t n, Counters* cnt, int accumulate) -> int {
    A.record = rec;
    A.path_base = p0;
    A.n_paths = n;
    A.accumulate = accumulate;
    A.nee.job = (float4*)ctx->L->ws[W_NEE_JOB].p;
    A.nee.jm = (uint32_t*)ctx->L->ws[W_NEE_JM].p;
    A.nee.jpath = (uint32_t*)ctx->L->ws[W_NEE_PATH].p;
    A.nee.jx = (float4*)ctx->L->ws[W_NEE_JX].p;
    A.nee.jw = (float4*)ctx->L->ws[W_NEE_JW].p;
    if (rec == (const uint32_t*)ctx->L->record.p) {  // a recorded pass kept its secondary-ray results
      A.nres.res = (float4*)ctx->L->ws[W_NEE_RES].p;
      A.nres.xo = (uint2*)ctx->L->ws[W_NEE_XO].p;
      A.nres.xing = (uint2*)ctx->L->ws[W_XING].p;
    } else {
      A.nres = NeeRes{};
    }
    A.cnt = cnt;
    CKS(ws(ctx, W_SEEDS, (size_t)n * K1, st, &A.seeds));
    const bool rnee = q.rough_nee && sc->rough;
    uint32_t rough_mask = 0u;
    A.seedv = nullptr;
    if (rnee) {
      CKS(ws(ctx, W_SEEDV, 2 * (size_t)n * K1, st, &A.seedv));
      for (int mi = 0; mi < med.M; ++mi)
        if (med.rough[mi] > 0.0f) rough_mask |= 1u << mi;
    }
    CKS(ws(ctx, W_ACTIVE, (size_t)n + 1, st, &active));
    CKS(ws(ctx, W_ACT_CNT, 64, st, &work));
    A.active = active;
    A.n_active = work + 51;
    uint8_t* pclass;
    CKS(ws(ctx, W_PCLASS, (size_t)n, st, &pclass));
    // the active-path lists (a pass over the record) do not depend on the secondary-ray
    // adjoint: on the lane's second stream they run beside it
    const bool nee_adj = (sc->dev.n_scat > 0 || rnee) && A.nee.job;
    const bool fork = nee_adj && ctx->opts[US_OPT_NEE_STREAM] > 0;
    Lane* L = ctx->L;
    cudaStream_t as = st;
    if (fork) {
      CKS(ensure_side(ctx, L));
      CK(cudaEventRecord(L->ev_afork, st));
      CK(cudaStreamWaitEvent(L->side, L->ev_afork, 0));
      as = L->side;
    }
    {
      StageScope sc_(ctx, US_STAGE_PATH_ADJ, 3, as);
      launch_active_paths(rec, n, q.kmax, work, pclass, active, grid_of(ctx, 4), as, rough_mask, sc->dev.tri_nrm);
    }
    if (nee_adj) {
      A.gpart = gpart + (size_t)grid * A.P;
      StageScope sc_(ctx, US_STAGE_NEE_ADJ, 1, st);
      launch_nee_adjoint(A, grid, st);
    } else if (!accumulate) {
      CK(cudaMemsetAsync(gpart + (size_t)grid * A.P, 0, sizeof(float) * grid * A.P, st));
    }
    if (fork) {
      CK(cudaEventRecord(L->ev_ajoin, L->side));
      CK(cudaStreamWaitEvent(st, L->ev_ajoin, 0));
    }
    {
      StageScope sc_(ctx, US_STAGE_PATH_ADJ, 1, st);
      A.gpart = gpart;
      launch_path_adjoint(A, grid, st);
    }
    return US_OK;
  };
  if (mode == 0) {
    if (!ctx->L->rkey.valid || ctx->L->rkey.scene != scene || ctx->L->rkey.seed != seed || ctx->L->rkey.n_paths != n_paths ||
        ctx->L->rkey.acq.size() != sizeof q || std::memcmp(ctx->L->rkey.acq.data(), &q, sizeof q) != 0 ||
        ctx->L->rkey.theta.size() != (size_t)Ps ||
        std::memcmp(ctx->L->rkey.theta.data(), theta, sizeof(float) * Ps) != 0)
      return fail(ctx, US_ERR_STATE, "record mode needs the last forward pass, with keep_record, on the same inputs");
    CKS(sweep((const uint32_t*)ctx->L->record.p, 0, (uint32_t)n_paths, (Counters*)ctx->L->ws[W_CNT].p, 0));
  } else {
    // recompute: regenerate the decisions chunk by chunk, then sweep each chunk
    const long long chunk = std::min<long long>(n_paths, 1ll << 22);
    uint32_t* rec;
    Counters* cnt;
    CKS(ws(ctx, W_REC_CHUNK, (size_t)chunk * K1, st, &rec));
    CKS(ws(ctx, W_CNT, 1, st, &cnt));
    ctx->L->rkey.valid = false;  // the job buffers and counters now hold the recomputed chunk
    for (long long p0 = 0; p0 < n_paths; p0 += chunk) {
      const uint32_t n = (uint32_t)std::min<long long>(chunk, n_paths - p0);
      CKS(run_transport(ctx, sc, med, q, p0, n, nullptr, 0, rec, false, cnt, st));
      CKS(sweep(rec, p0, n, cnt, p0 > 0));
    }
  }
  {
    StageScope sc_(ctx, US_STAGE_PATH_ADJ, 1, st);
    launch_grad_reduce_split(gpart, 2 * grid, A.P, Ps, dL_dtheta_dev, dL_dacq_dev, acc_acq, st);
  }
  CK(cudaGetLastError());
  return US_OK;
}

int us_transport_vjp(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, uint64_t seed,
                     int mode, const float* dL_drf_dev, float* dL_dtheta_dev, void* stream) {
  return transport_vjp(ctx, scene, theta, acq, seed, mode, dL_drf_dev, dL_dtheta_dev, nullptr, 0, stream);
}

int us_transport_vjp_acq(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, uint64_t seed,
                         int mode, const float* dL_drf_dev, float* dL_dtheta_dev, float* dL_dacq_dev, void* stream) {
  if (ctx && !dL_dacq_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  return transport_vjp(ctx, scene, theta, acq, seed, mode, dL_drf_dev, dL_dtheta_dev, dL_dacq_dev, 0, stream);
}

int us_transport_vjp_shape(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, uint64_t seed,
                           int mode, const float* dL_drf_dev, float* dL_dtheta_dev, float* dL_dtris_dev,
                           void* stream) {
  if (ctx && !dL_dtris_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  return transport_vjp(ctx, scene, theta, acq, seed, mode, dL_drf_dev, dL_dtheta_dev, nullptr, 0, stream,
                       dL_dtris_dev);
}

int us_shape_param_grad(us_ctx* ctx, int64_t n_tris, const float* dL_dtris_dev, int n_param, const float* dtris_dq_dev,
                        float* dL_dq_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  if (n_tris < 0 || n_param < 1 || n_param > 65535 || !dL_dtris_dev || !dtris_dq_dev || !dL_dq_dev)
    return fail(ctx, US_ERR_ARG, "invalid arguments");
  StageScope sc_(ctx, US_STAGE_OTHER, 1, (cudaStream_t)stream);
  launch_tangent_dot(9 * n_tris, dL_dtris_dev, n_param, dtris_dq_dev, dL_dq_dev, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return US_OK;
}

// S7' (DAS derivative in the acquisition parameters) contracted with dL/dI_rf; acc: add
static int das_acq_vjp(us_ctx* ctx, const Acq& q, const Img& im, const float* rf_dev, const float* gi_dev,
                       float* dL_dacq_dev, int acc, cudaStream_t st) {
  float* part;
  const int nb = das_acq_blocks(im);
  CKS(ws(ctx, W_ACQ_PART, (size_t)nb * (2 + q.ntx), st, &part));
  StageScope sc_(ctx, US_STAGE_DAS_ACQ, 2, st);
  launch_das_acq(q, im, rf_dev, gi_dev, part, st);
  launch_grad_reduce_split(part, nb, 2 + q.ntx, 0, nullptr, dL_dacq_dev, acc, st);
  CK(cudaGetLastError());
  return US_OK;
}

int us_das_acq_vjp(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev,
                   const float* dL_dirf_dev, float* dL_dacq_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  Acq q;
  Img im;
  CKS(make_acq(ctx, acq, 0, q));
  CKS(make_img(ctx, img, im));
  if (!rf_dev || !dL_dirf_dev || !dL_dacq_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  return das_acq_vjp(ctx, q, im, rf_dev, dL_dirf_dev, dL_dacq_dev, 0, (cudaStream_t)stream);
}

int us_adjoint(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, const us_img_desc* img,
               uint64_t seed, int mode, const float* rf_dev, const float* dL_dB_dev, float* dL_dtheta_dev,
               float* dL_drf_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Acq q;
  CKS(make_acq(ctx, acq, seed, q));
  float* grf = dL_drf_dev;
  if (!grf) CKS(ws(ctx, W_GRF, (size_t)q.ntx * q.ne * q.ns, st, &grf));
  CKS(bmode_vjp(ctx, acq, img, rf_dev, dL_dB_dev, grf, stream, mode == 0));
  return us_transport_vjp(ctx, scene, theta, acq, seed, mode, grf, dL_dtheta_dev, stream);
}

int us_adjoint_shape(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, const us_img_desc* img,
                     uint64_t seed, int mode, const float* rf_dev, const float* dL_dB_dev, float* dL_dtheta_dev,
                     float* dL_dtris_dev, float* dL_drf_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!dL_dtris_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  Acq q;
  CKS(make_acq(ctx, acq, seed, q));
  float* grf = dL_drf_dev;
  if (!grf) CKS(ws(ctx, W_GRF, (size_t)q.ntx * q.ne * q.ns, st, &grf));
  CKS(bmode_vjp(ctx, acq, img, rf_dev, dL_dB_dev, grf, stream, mode == 0));
  return transport_vjp(ctx, scene, theta, acq, seed, mode, grf, dL_dtheta_dev, nullptr, 0, stream, dL_dtris_dev);
}

int us_adjoint_acq(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, const us_img_desc* img,
                   uint64_t seed, int mode, const float* rf_dev, const float* dL_dB_dev, float* dL_dtheta_dev,
                   float* dL_dacq_dev, float* dL_drf_dev, void* stream) {
  if (!ctx) return US_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!dL_dacq_dev) return fail(ctx, US_ERR_ARG, "null buffer");
  Acq q;
  Img im;
  CKS(make_acq(ctx, acq, seed, q));
  CKS(make_img(ctx, img, im));
  float* grf = dL_drf_dev;
  if (!grf) CKS(ws(ctx, W_GRF, (size_t)q.ntx * q.ne * q.ns, st, &grf));
  CKS(bmode_vjp(ctx, acq, img, rf_dev, dL_dB_dev, grf, stream, mode == 0));
  // dL/dI_rf is left in the lane's W_GI workspace by bmode_vjp
  CKS(das_acq_vjp(ctx, q, im, rf_dev, (const float*)ctx->L->ws[W_GI].p, dL_dacq_dev, 0, st));
  return transport_vjp(ctx, scene, theta, acq, seed, mode, grf, dL_dtheta_dev, dL_dacq_dev, 1, stream);
}

// -----------------------------------------------------------------------------------------
// Batches: requests spread round-robin over lanes; each lane runs its requests in order on
// its own stream, forked from and joined back to the caller's stream, so a whole batch is one
// stream-ordered unit that can be captured in a CUDA graph (after one call outside capture
// has grown the lanes' workspaces).
// -----------------------------------------------------------------------------------------
static int run_request(us_ctx* ctx, const us_request& r, cudaStream_t st) {
  CKS(us_forward(ctx, r.scene, r.theta, r.acq, r.img, r.seed, r.bref_dev != nullptr, r.rf_dev, r.bmode_dev, st));
  if (r.bref_dev) {
    if (!r.bmode_dev || !r.loss_dev || !r.dL_dtheta_dev)
      return fail(ctx, US_ERR_ARG, "a forward+adjoint request needs bmode_dev, loss_dev and dL_dtheta_dev");
    Img im;
    CKS(make_img(ctx, r.img, im));
    float* gb;
    CKS(ws(ctx, W_GB, (size_t)im.nl * im.nd, st, &gb));
    CKS(us_loss(ctx, r.img, r.bmode_dev, r.bref_dev, r.loss_dev, gb, st));
    CKS(us_adjoint(ctx, r.scene, r.theta, r.acq, r.img, r.seed, 0, r.rf_dev, gb, r.dL_dtheta_dev, nullptr, st));
  }
  return US_OK;
}

int us_forward_batch(us_ctx* ctx, int n, const us_request* reqs, void* stream) {
  if (!ctx || n < 0 || (n && !reqs)) return fail(ctx, US_ERR_ARG, "invalid batch");
  cudaStream_t st = (cudaStream_t)stream;
  const int nl = std::max(1, std::min(ctx->opts[US_OPT_LANES], 16));
  while ((int)ctx->lanes.size() < nl + 1)
    if (!new_lane(ctx, true)) return fail(ctx, US_ERR_CUDA, "cannot create a lane stream");
  Lane* lane0 = ctx->lanes[0];
  // fork: every lane waits for the work already on the caller's stream
  CK(cudaEventRecord(lane0->ev_done, st));
  for (int i = 1; i <= nl; ++i) CK(cudaStreamWaitEvent(ctx->lanes[i]->stream, lane0->ev_done, 0));
  int rc = US_OK;
  for (int j = 0; j < n && rc == US_OK; ++j) {
    Lane* l = ctx->lanes[1 + j % nl];
    ctx->L = l;
    rc = run_request(ctx, reqs[j], l->stream);
  }
  ctx->L = lane0;
  // join: the caller's stream waits for every lane
  for (int i = 1; i <= nl; ++i) {
    CK(cudaEventRecord(ctx->lanes[i]->ev_done, ctx->lanes[i]->stream));
    CK(cudaStreamWaitEvent(st, ctx->lanes[i]->ev_done, 0));
  }
  return rc;
}

int us_run_request(us_ctx* ctx, int lane, const us_request* req, void* stream) {
  if (!ctx || !req || lane < 1 || lane > 16) return fail(ctx, US_ERR_ARG, "lane must lie in [1, 16]");
  while ((int)ctx->lanes.size() <= lane)
    if (!new_lane(ctx, true)) return fail(ctx, US_ERR_CUDA, "cannot create a lane");
  Lane* lane0 = ctx->lanes[0];
  ctx->L = ctx->lanes[lane];
  const int rc = run_request(ctx, *req, (cudaStream_t)stream);
  ctx->L = lane0;
  return rc;
}

int us_request_bytes(us_ctx* ctx, const us_request* req, size_t* bytes) {
  if (!ctx || !req || !bytes) return fail(ctx, US_ERR_ARG, "null argument");
  Acq q;
  CKS(make_acq(ctx, req->acq, 0, q));
  const size_t n = (size_t)(q.rays_per_tx * q.ntx), K1 = q.kmax + 1, jobs = n * std::max(1, q.kmax);
  size_t b = n * (2 * 48 + 8 + 2 * 4) + jobs * 2 * 24 + n * K1 * 16 * 2;  // queues, hits, ray and job keys,
                                                                          // jobs, arrivals
  if (req->bref_dev) b += n * K1 * (4 + 8) + n * 4 + jobs * (16 + 8 + 16);  // record, seeds, active list,
                                                                               // secondary-ray results
  if (req->img) b += (size_t)req->img->n_lines * req->img->n_depth * 4 * 5;
  b += (size_t)q.ntx * q.ne * q.ns * (req->bref_dev ? 4 + 8 : 4);       // dL/dRF (and its fixed-point sums)
  *bytes = b;
  return US_OK;
}

int us_autotune_batch(us_ctx* ctx, int n, const us_request* reqs, void* stream, int* best_lanes,
                      int* best_trav_per_sm) {
  if (!ctx || n < 1 || !reqs) return fail(ctx, US_ERR_ARG, "invalid batch");
  cudaStream_t st = (cudaStream_t)stream;
  const int base_trav = traverse_blocks_per_sm() / 2;  // resident blocks of the traversal kernel
  const int lane_opts[] = {1, 2, 4, 8};
  const int trav_opts[] = {1, 2, 4};
  float best = 3.0e38f;
  int bl = ctx->opts[US_OPT_LANES], bt = ctx->trav_per_sm;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int lo : lane_opts)
    for (int to : trav_opts) {
      ctx->opts[US_OPT_LANES] = lo;
      ctx->trav_per_sm = base_trav * to;
      CKS(us_forward_batch(ctx, n, reqs, stream));  // warm-up: grows the lanes' workspaces
      CK(cudaEventRecord(e0, st));
      CKS(us_forward_batch(ctx, n, reqs, stream));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bl = lo;
        bt = ctx->trav_per_sm;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->opts[US_OPT_LANES] = bl;
  ctx->trav_per_sm = bt;
  if (best_lanes) *best_lanes = bl;
  if (best_trav_per_sm) *best_trav_per_sm = bt;
  return US_OK;
}

}  // extern "C"
