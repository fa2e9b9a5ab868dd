// Serving: continuous batching of BC requests over the context's resident graphs.
//
// bc_stream_submit queues a request (a source list, or k sources drawn from a seed) and
// returns at once.  Worker threads (one CUDA stream each) repeatedly
//   * admit queued requests in arrival order while their device footprint (a BC
//     accumulator of n doubles, plus the graph's tile workspace the first time the graph
//     is served) fits the context's HBM budget;
//   * pick a graph that has unscheduled sources and is not being run by another worker,
//     fill one tile with up to T sources taken from that graph's admitted requests in
//     admission order (sources of several requests share the tile; each lane's
//     dependencies are routed to its own request's accumulator);
//   * run the tile with per-phase launches (not the cooperative kernel) so that tiles of
//     different graphs, on different streams, overlap on the device;
//   * on graphs the autotuner gave to the per-source path (untuned: up to 65,536 vertices),
//     instead run the remaining sources of all the graph's admitted requests (up to
//     kCtaMaxReq) in one call of the per-source CTA kernel, each request on CTAs of its
//     own (each CTA a source at a time), which there is far faster than a tile;
//   * complete a request when its last tile is done: copy its BC to the caller's buffer.
// A request that arrives while others run is admitted as soon as memory allows and its
// sources join the next tiles of its graph.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "bc_internal.h"

namespace bcl {

uint64_t splitmix64_next(uint64_t &x);
std::vector<int64_t> sample_distinct(int64_t N, int64_t k, uint64_t seed);
bc_status nonisolated_host(Graph *g, std::vector<int32_t> &out);

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kWorkers = 4;
constexpr int kMaxReqPerTile = 8;
// request-buffer pointers per graph: a tile's requests or a per-CTA launch's
constexpr int kReqPtrs = kCtaMaxReq > kMaxReqPerTile ? kCtaMaxReq : kMaxReqPerTile;

struct Req {
  uint64_t id = 0;
  Graph *g = nullptr;
  std::vector<int32_t> src;
  double *h_out = nullptr;
  double scale = 1.0;
  Clock::time_point t_submit, t_start;
  bool started = false, admitted = false, canceled = false, done = false;
  double queue_s = 0.0, latency_s = 0.0;
  bc_status status = BC_OK;
  double *d_bc = nullptr;
  size_t next = 0;
  int inflight = 0;
};

struct GraphExec {
  Graph *g = nullptr;
  TileWS *ws = nullptr;
  CtaWS *cta = nullptr;        // small graphs: per-source CTA kernel workspace
  int32_t *d_many = nullptr;   // its source list
  size_t cap_many = 0;
  int32_t *d_src = nullptr;
  uint8_t *d_lane = nullptr;
  double **d_reqbc = nullptr;
  bool busy = false;
  bool counted = false;
  bool keys_tried = false;      // tiles: landmark profiles looked up (host copy)
  const uint8_t *keys = nullptr;  // [n][nkeys] distances to the landmarks, or null
  int nkeys = 0;
};

// Tiles are cut from the pending sources of a graph's oldest requests, up to this many
// tiles' worth, grouped by their landmark profiles.
constexpr int kOrderWindow = 16;

}  // namespace

struct Server {
  Ctx *ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_id = 1;
  std::map<uint64_t, Req *> reqs;
  std::deque<Req *> pending;
  std::vector<Req *> active;
  std::map<Graph *, GraphExec *> gx;
  std::vector<std::thread> workers;
};

namespace {

// Kernel of a graph's requests: the autotuner's choice when the graph was tuned (the per-CTA
// kernel when it picked the per-source path, tiles otherwise), else by size (per-CTA up to
// 65,536 vertices).
bool serve_on_cta(const Graph *g) {
  if (g->tune.ready)
    return g->tune.res.tile_width == 0 && (g->tune.res.plain_cta || cta_fits(g->g.n)) &&
           g->g.n <= kCtaForcedMaxN;
  return cta_fits(g->g.n);
}

int tile_width_for(Graph *g) {
  if (g->tune.ready && g->tune.res.tile_width > 0) return g->tune.res.tile_width;
  return 64;
}

size_t tile_ws_estimate(Graph *g, int T) {
  const size_t n = (size_t)g->g.n, G = (size_t)T / 32;
  if (serve_on_cta(g)) return n * 64;  // CTA kernel: it shrinks its partials to the budget
  return n * G * 20 + n * T * 16 + n * (20 + 12 * G) * 4;
}

void exec_release(Ctx *c, GraphExec *e) {
  if (e->ws) tile_free(c, e->ws);
  if (e->cta) cta_free(c, e->cta);
  if (e->d_many) c->mem.release(e->d_many, e->cap_many * 4);
  if (e->d_src) c->mem.release(e->d_src, 256 * 4);
  if (e->d_lane) c->mem.release(e->d_lane, 256);
  if (e->d_reqbc) c->mem.release(e->d_reqbc, kReqPtrs * sizeof(double *));
}

// Frees a graph's cached workspaces (it has no request running); they are rebuilt on its next
// request.
void exec_trim(Ctx *c, GraphExec *e) {
  exec_release(c, e);
  e->ws = nullptr;
  e->cta = nullptr;
  e->d_many = nullptr;
  e->cap_many = 0;
  e->d_src = nullptr;
  e->d_lane = nullptr;
  e->d_reqbc = nullptr;
  e->counted = false;
}

void finish(Server *sv, Req *r, bc_status st) {
  Ctx *c = sv->ctx;
  if (st == BC_OK && !r->canceled && r->d_bc && !r->src.empty()) {
    cudaError_t e = cudaMemcpy(r->h_out, r->d_bc, (size_t)r->g->g.n * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_fail(e, "serving: copy of the result");
  } else if (st == BC_OK && !r->canceled && r->src.empty()) {
    memset(r->h_out, 0, (size_t)r->g->g.n * 8);
  }
  if (r->d_bc) c->mem.release(r->d_bc, (size_t)r->g->g.n * 8);
  r->d_bc = nullptr;
  r->status = r->canceled ? BC_ECANCELED : st;
  r->latency_s = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
  if (!r->started) r->queue_s = r->latency_s;
  r->done = true;
  sv->active.erase(std::remove(sv->active.begin(), sv->active.end(), r), sv->active.end());
  r->g->inflight--;
  sv->cv_done.notify_all();
}

// Admission in arrival order while the footprint fits.  Caller holds sv->mu.
void admit(Server *sv) {
  Ctx *c = sv->ctx;
  while (!sv->pending.empty()) {
    Req *r = sv->pending.front();
    size_t need = (size_t)r->g->g.n * 8;
    auto it = sv->gx.find(r->g);
    const bool ws_counted = it != sv->gx.end() && it->second->counted;
    if (!ws_counted) need += tile_ws_estimate(r->g, tile_width_for(r->g));
    bool fits = c->mem.budget == 0 || c->mem.used.load() + need <= c->mem.budget;
    if (!fits && !sv->active.empty()) return;  // wait for memory to free up
    if (!fits) {  // nothing runs: the cached workspaces of idle graphs give their memory back
      for (auto &kv : sv->gx)
        if (!kv.second->busy) exec_trim(c, kv.second);
      need = (size_t)r->g->g.n * 8 + tile_ws_estimate(r->g, tile_width_for(r->g));
      fits = c->mem.used.load() + need <= c->mem.budget;
    }
    if (!fits) {
      sv->pending.pop_front();
      finish(sv, r, fail(BC_ENOMEM, "serving: request does not fit the context HBM budget"));
      continue;
    }
    bc_status s = c->mem.alloc((void **)&r->d_bc, (size_t)r->g->g.n * 8);
    if (s == BC_ENOMEM && c->mem.budget) {  // a worker's workspace took the room meanwhile
      if (!sv->active.empty()) return;       // wait for memory to free up
      for (auto &kv : sv->gx)
        if (!kv.second->busy) exec_trim(c, kv.second);
      s = c->mem.alloc((void **)&r->d_bc, (size_t)r->g->g.n * 8);
    }
    sv->pending.pop_front();
    // zeroed before a worker's stream (non-blocking, so unordered with this one) adds to it
    if (!s && (cudaMemsetAsync(r->d_bc, 0, (size_t)r->g->g.n * 8, nullptr) != cudaSuccess ||
               cudaStreamSynchronize(nullptr) != cudaSuccess))
      s = fail(BC_ECUDA, "serving: clearing a request's result buffer");
    r->admitted = true;
    sv->active.push_back(r);
    if (s || r->src.empty()) {
      finish(sv, r, s);
      continue;
    }
  }
}

GraphExec *exec_for(Server *sv, Graph *g) {
  auto it = sv->gx.find(g);
  if (it != sv->gx.end()) return it->second;
  GraphExec *e = new GraphExec();
  e->g = g;
  sv->gx[g] = e;
  return e;
}

bc_status exec_buffers(Ctx *c, GraphExec *e) {
  if (e->d_src) return BC_OK;
  bc_status s = c->mem.alloc((void **)&e->d_src, 256 * 4);
  if (!s) s = c->mem.alloc((void **)&e->d_lane, 256);
  if (!s) s = c->mem.alloc((void **)&e->d_reqbc, kReqPtrs * sizeof(double *));
  return s;
}

struct Cand {
  const uint8_t *key;  // the source's landmark profile
  int ri, pos;         // request (index in the window) and position in its source list
};

void mark_started(Req *r) {
  if (!r->started) {
    r->started = true;
    r->t_start = Clock::now();
    r->queue_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
  }
}

// One tile of graph g from the pending sources of its oldest requests (at most kOrderWindow
// tiles' worth), sorted by landmark profile: the T sources nearest in that order to the
// oldest request's next source (so that request always advances), from at most
// kMaxReqPerTile requests.  Each request's taken sources move to the front of its pending
// part; lanes are grouped by request.
void select_by_locality(Server *sv, Graph *g, const uint8_t *keys, int L, int T, std::vector<Cand> &cand,
                        std::vector<std::pair<int, int>> &chosen, std::vector<int32_t> &hsrc,
                        std::vector<uint8_t> &hlane, std::vector<double *> &hreq,
                        std::vector<std::pair<Req *, int>> &slots) {
  std::vector<Req *> rq;
  cand.clear();
  chosen.clear();
  for (Req *r : sv->active) {
    if (r->g != g || r->canceled || r->next >= r->src.size()) continue;
    if (!rq.empty() && cand.size() >= (size_t)kOrderWindow * T) break;
    const int ri = (int)rq.size();
    rq.push_back(r);
    for (size_t i = r->next; i < r->src.size(); i++)
      cand.push_back(Cand{keys + (size_t)r->src[i] * L, ri, (int)i});
  }
  if (rq.empty()) return;
  std::sort(cand.begin(), cand.end(), [L](const Cand &a, const Cand &b) {
    const int c = memcmp(a.key, b.key, (size_t)L);
    if (c != 0) return c < 0;
    return a.ri != b.ri ? a.ri < b.ri : a.pos < b.pos;
  });
  int a = 0;
  while (!(cand[a].ri == 0 && cand[a].pos == (int)rq[0]->next)) a++;
  std::vector<int> used;  // requests in the tile
  auto take = [&](int i) {
    const int ri = cand[i].ri;
    if (std::find(used.begin(), used.end(), ri) == used.end()) {
      if ((int)used.size() >= kMaxReqPerTile) return;
      used.push_back(ri);
    }
    chosen.emplace_back(ri, cand[i].pos);
  };
  take(a);
  for (int l = a - 1, h = a + 1; (int)chosen.size() < T && (l >= 0 || h < (int)cand.size());) {
    if (h < (int)cand.size()) take(h++);
    if ((int)chosen.size() < T && l >= 0) take(l--);
  }
  std::sort(chosen.begin(), chosen.end());
  for (size_t i = 0; i < chosen.size();) {
    const int ri = chosen[i].first;
    Req *r = rq[(size_t)ri];
    const uint8_t slot = (uint8_t)slots.size();
    const size_t first = r->next;
    for (; i < chosen.size() && chosen[i].first == ri; i++) {
      std::swap(r->src[r->next], r->src[(size_t)chosen[i].second]);
      r->next++;
    }
    for (size_t j = first; j < r->next; j++) {
      hsrc.push_back(r->src[j]);
      hlane.push_back(slot);
    }
    r->inflight++;
    mark_started(r);
    hreq.push_back(r->d_bc);
    slots.emplace_back(r, (int)(r->next - first));
  }
}

void worker_main(Server *sv, int wid) {
  Ctx *c = sv->ctx;
  cudaSetDevice(c->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<int32_t> hsrc;
  std::vector<uint8_t> hlane;
  std::vector<double *> hreq;
  std::vector<std::pair<Req *, int>> slots;
  std::vector<int32_t> hk;
  std::vector<Cand> cand;
  std::vector<std::pair<int, int>> chosen;
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    admit(sv);
    // a graph with unscheduled sources that no other worker is running
    GraphExec *job = nullptr;
    for (Req *r : sv->active) {
      if (r->canceled || r->next >= r->src.size()) continue;
      GraphExec *e = exec_for(sv, r->g);
      if (!e->busy) {
        job = e;
        break;
      }
    }
    if (!job) {
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    Graph *g = job->g;
    if (serve_on_cta(g)) {
      // small graph (or one the autotuner gave to the per-CTA kernel): the remaining sources
      // of up to kCtaMaxReq of its admitted requests, in admission order, in one call; each
      // request gets CTAs of its own, so requests that arrived while the last call ran share
      // the next one instead of waiting for one call each
      hsrc.clear();
      hreq.clear();
      hk.clear();
      slots.clear();
      for (Req *q : sv->active) {
        if ((int)slots.size() >= kCtaMaxReq) break;
        if (q->g != g || q->canceled || q->next >= q->src.size()) continue;
        const int take = (int)(q->src.size() - q->next);
        hsrc.insert(hsrc.end(), q->src.begin() + (long)q->next, q->src.end());
        q->next = q->src.size();
        q->inflight++;
        if (!q->started) {
          q->started = true;
          q->t_start = Clock::now();
          q->queue_s = std::chrono::duration<double>(q->t_start - q->t_submit).count();
        }
        hk.push_back(take);
        hreq.push_back(q->d_bc);
        slots.emplace_back(q, take);
      }
      const size_t k = hsrc.size();
      job->busy = true;
      job->counted = true;
      lk.unlock();
      bc_status s = exec_buffers(c, job);
      if (!s && job->cap_many < k) {
        if (job->d_many) c->mem.release(job->d_many, job->cap_many * 4);
        job->d_many = nullptr;
        job->cap_many = 0;
        s = c->mem.alloc((void **)&job->d_many, k * 4);
        if (!s) job->cap_many = k;
      }
      if (!s && cudaMemcpyAsync(job->d_many, hsrc.data(), k * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        s = fail(BC_ECUDA, "serving: copy of request sources");
      if (!s && cudaMemcpyAsync(job->d_reqbc, hreq.data(), hreq.size() * sizeof(double *), cudaMemcpyHostToDevice,
                                st) != cudaSuccess)
        s = fail(BC_ECUDA, "serving: copy of request buffers");
      if (!s) {
        PlainArgs pa{};
        pa.g = &g->g;
        pa.src = job->d_many;
        pa.nsrc = (int32_t)k;
        pa.max_degree = g->max_degree;
        pa.nreq = (int32_t)slots.size();
        pa.h_req_k = hk.data();
        pa.req_bc = job->d_reqbc;
        s = cta_run(c, g, &job->cta, pa, st, nullptr);
      }
      lk.lock();
      job->busy = false;
      for (auto &sl : slots) {
        Req *q = sl.first;
        q->inflight--;
        if (s && q->status == BC_OK) q->status = s;
        if (q->inflight == 0) finish(sv, q, q->status);
      }
      sv->cv_work.notify_all();
      continue;
    }
    const int T = tile_width_for(g);
    if (!job->keys_tried) {  // the graph's landmark profiles (once; the graph stays ours)
      job->busy = true;
      lk.unlock();
      const uint8_t *keys = nullptr;
      int nkeys = 0;
      {
        std::lock_guard<std::mutex> glk(g->mu);
        if (order_host_keys(g, &g->g, T, st, &job->ws, &keys, &nkeys) != BC_OK) {
          keys = nullptr;  // tiles in admission order instead
          nkeys = 0;
        }
      }
      lk.lock();
      job->keys = keys;
      job->nkeys = nkeys;
      job->keys_tried = true;
    }
    hsrc.clear();
    hlane.clear();
    hreq.clear();
    slots.clear();
    if (job->keys) {
      select_by_locality(sv, g, job->keys, job->nkeys, T, cand, chosen, hsrc, hlane, hreq, slots);
    } else for (Req *r : sv->active) {
      if ((int)hsrc.size() >= T || (int)slots.size() >= kMaxReqPerTile) break;
      if (r->g != g || r->canceled || r->next >= r->src.size()) continue;
      const int take = (int)std::min<size_t>((size_t)(T - (int)hsrc.size()), r->src.size() - r->next);
      const uint8_t slot = (uint8_t)slots.size();
      for (int i = 0; i < take; i++) {
        hsrc.push_back(r->src[r->next + i]);
        hlane.push_back(slot);
      }
      r->next += take;
      r->inflight++;
      if (!r->started) {
        r->started = true;
        r->t_start = Clock::now();
        r->queue_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
      }
      hreq.push_back(r->d_bc);
      slots.emplace_back(r, take);
    }
    job->busy = true;
    if (!job->counted) {
      job->counted = true;  // the workspace is accounted by tile_run's own allocations
    }
    lk.unlock();
    bc_status s = exec_buffers(c, job);
    if (!s && cudaMemcpyAsync(job->d_src, hsrc.data(), hsrc.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      s = fail(BC_ECUDA, "serving: copy of tile sources");
    if (!s && cudaMemcpyAsync(job->d_lane, hlane.data(), hlane.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
      s = fail(BC_ECUDA, "serving: copy of lane slots");
    if (!s && cudaMemcpyAsync(job->d_reqbc, hreq.data(), hreq.size() * sizeof(double *), cudaMemcpyHostToDevice, st) != cudaSuccess)
      s = fail(BC_ECUDA, "serving: copy of request buffers");
    if (!s) {
      TileArgs ta{};
      ta.g = &g->g;
      ta.src = job->d_src;
      ta.nsrc = (int32_t)hsrc.size();
      ta.bc = nullptr;
      ta.T = T;
      ta.loop_mode = 1;
      ta.alpha = g->tune.ready ? g->tune.res.alpha : 0.2f;
      if (g->tune.ready && g->tune.res.tile_width > 0) {  // the tuned tile thresholds
        ta.beta = g->tune.res.beta;
        ta.hub = g->tune.res.hub_degree;
        ta.hub_chunk = g->tune.res.hub_chunk;
      }
      ta.nreq = (int32_t)slots.size();
      ta.lane_req = job->d_lane;
      ta.req_bc = job->d_reqbc;
      s = tile_run(c, g, &job->ws, ta, st, nullptr);
    }
    lk.lock();
    job->busy = false;
    for (auto &sl : slots) {
      Req *r = sl.first;
      r->inflight--;
      if (s && r->status == BC_OK) r->status = s;
      if (r->inflight == 0 && (r->next >= r->src.size() || r->canceled || r->status != BC_OK))
        finish(sv, r, r->status);
    }
    sv->cv_work.notify_all();
  }
  lk.unlock();
  if (st) cudaStreamDestroy(st);
  (void)wid;
}

Server *server_get(Ctx *c) {
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->server) {
    Server *sv = new Server();
    sv->ctx = c;
    c->server = sv;
    for (int i = 0; i < kWorkers; i++) sv->workers.emplace_back(worker_main, sv, i);
  }
  return c->server;
}

Ctx *ctx_of(bc_ctx *h) {
  Ctx *c = (Ctx *)h;
  return (c && c->magic == kCtxMagic) ? c : nullptr;
}

}  // namespace

void server_stop(Ctx *c) {
  Server *sv = nullptr;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    sv = c->server;
    c->server = nullptr;
  }
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto &t : sv->workers) t.join();
  for (auto &kv : sv->reqs) {
    Req *r = kv.second;
    if (r->d_bc) c->mem.release(r->d_bc, (size_t)r->g->g.n * 8);
    delete r;
  }
  for (auto &kv : sv->gx) {
    exec_release(c, kv.second);
    delete kv.second;
  }
  delete sv;
}

bool server_graph_busy(Ctx *c, Graph *g) {
  Server *sv;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    sv = c->server;
  }
  if (!sv) return false;
  std::lock_guard<std::mutex> lk(sv->mu);
  for (auto &kv : sv->reqs)
    if (kv.second->g == g && !kv.second->done) return true;
  return false;
}

// Release the serving state kept for a graph that is being destroyed.
void server_forget_graph(Ctx *c, Graph *g) {
  Server *sv;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    sv = c->server;
  }
  if (!sv) return;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->gx.find(g);
  if (it == sv->gx.end()) return;
  GraphExec *e = it->second;
  exec_release(c, e);
  delete e;
  sv->gx.erase(it);
  for (auto it2 = sv->reqs.begin(); it2 != sv->reqs.end();) {  // finished, unpolled results
    if (it2->second->g == g) {
      delete it2->second;
      it2 = sv->reqs.erase(it2);
    } else {
      ++it2;
    }
  }
}

}  // namespace bcl

using namespace bcl;

extern "C" bc_status bc_stream_submit(bc_ctx *ctx, const bc_request *req, uint64_t *request_id) {
  Ctx *c = ctx_of(ctx);
  if (!c || !req || !request_id) return fail(BC_EINVAL, "bc_stream_submit: NULL argument");
  Graph *g = (Graph *)req->graph;
  if (!g || g->magic != kGraphMagic || g->ctx != c)
    return fail(BC_EINVAL, "bc_stream_submit: graph is not a graph of this context");
  if (!req->bc_out) return fail(BC_EINVAL, "bc_stream_submit: bc_out is NULL");
  if (req->k < 0) return fail(BC_EINVAL, "bc_stream_submit: k < 0");
  Req *r = new (std::nothrow) Req();
  if (!r) return fail(BC_ENOMEM, "bc_stream_submit: host allocation failed");
  r->g = g;
  r->h_out = req->bc_out;
  if (req->mode == BC_REQ_EXACT_LIST) {
    if (req->k > 0 && !req->src) {
      delete r;
      return fail(BC_EINVAL, "bc_stream_submit: src is NULL");
    }
    r->src.assign(req->src, req->src + req->k);
    for (int32_t v : r->src)
      if (v < 0 || v >= g->g.n) {
        delete r;
        return fail(BC_EINVAL, "bc_stream_submit: source id out of range");
      }
  } else if (req->mode == BC_REQ_SAMPLED) {
    std::vector<int32_t> pool;
    {
      std::lock_guard<std::mutex> lk(g->mu);
      cudaSetDevice(c->device);
      bc_status s = nonisolated_host(g, pool);
      if (s) {
        delete r;
        return s;
      }
    }
    if ((size_t)req->k > pool.size()) {
      delete r;
      return fail(BC_EINVAL, "bc_stream_submit: k exceeds the number of non-isolated vertices");
    }
    std::vector<int64_t> idx = sample_distinct((int64_t)pool.size(), req->k, req->seed);
    r->src.resize(idx.size());
    for (size_t i = 0; i < idx.size(); i++) r->src[i] = pool[(size_t)idx[i]];
    r->scale = req->k > 0 ? (double)pool.size() / (double)req->k : 1.0;
  } else {
    delete r;
    return fail(BC_EINVAL, "bc_stream_submit: unknown mode");
  }
  Server *sv = server_get(c);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    r->t_submit = Clock::now();
    g->inflight++;
    sv->reqs[r->id] = r;
    sv->pending.push_back(r);
    *request_id = r->id;
  }
  sv->cv_work.notify_all();
  return BC_OK;
}

extern "C" bc_status bc_stream_poll(bc_ctx *ctx, uint64_t request_id, int32_t timeout_us,
                                    bc_result *res) {
  Ctx *c = ctx_of(ctx);
  if (!c || !res) return fail(BC_EINVAL, "bc_stream_poll: NULL argument");
  Server *sv;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    sv = c->server;
  }
  if (!sv) return fail(BC_ENOTFOUND, "bc_stream_poll: unknown request id");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return fail(BC_ENOTFOUND, "bc_stream_poll: unknown request id");
  Req *r = it->second;
  if (!r->done && timeout_us != 0) {
    if (timeout_us < 0)
      sv->cv_done.wait(lk, [&] { return r->done; });
    else
      sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; });
  }
  if (!r->done) return fail(BC_EAGAIN, "bc_stream_poll: request still running");
  res->status = r->status;
  res->queue_seconds = r->queue_s;
  res->latency_seconds = r->latency_s;
  res->scale = r->scale;
  res->sources = (int64_t)r->src.size();
  sv->reqs.erase(it);
  delete r;
  return BC_OK;
}

extern "C" bc_status bc_stream_cancel(bc_ctx *ctx, uint64_t request_id) {
  Ctx *c = ctx_of(ctx);
  if (!c) return fail(BC_EINVAL, "bc_stream_cancel: bad context");
  Server *sv;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    sv = c->server;
  }
  if (!sv) return fail(BC_ENOTFOUND, "bc_stream_cancel: unknown request id");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return fail(BC_ENOTFOUND, "bc_stream_cancel: unknown request id");
  Req *r = it->second;
  if (r->done) return BC_OK;
  r->canceled = true;
  if (!r->admitted) {
    sv->pending.erase(std::remove(sv->pending.begin(), sv->pending.end(), r), sv->pending.end());
    finish(sv, r, BC_ECANCELED);
  } else if (r->inflight == 0) {
    finish(sv, r, BC_ECANCELED);
  }
  return BC_OK;
}
