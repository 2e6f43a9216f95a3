// sv_api.cu — host side of libsv.so: the C ABI declared in include/sv.h.
//
// Memory: the caller's device buffer is the pool (2 MiB pages, first fit). A compressed
// state owns a metadata run (device scalars, two block tables, per-block verbatim sums,
// tree scratch) and two arenas (ping-pong: a pass reads one and bump-allocates its output
// streams in the other). An arena that overflows during a pass poisons the state on the
// device (later passes return at once); sv_sync grows the arena to the size the pass asked
// for and replays the logged passes from the failed one, whose input arena is intact.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/sv.h"
#include "sv_internal.h"
#include "sv_tc.cuh"

using namespace sv;

namespace {

constexpr size_t kPage = 2u << 20;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct sv_pool {
  uint8_t* base = nullptr;  // device-accessible address of the buffer
  size_t bytes = 0;
  bool host = false;        // pinned host memory (a spill pool), reached over NVLink-C2C
  std::map<size_t, size_t> free_runs;  // offset -> length (bytes, page multiples)
  size_t used = 0;
  int nstates = 0;
  std::mutex mu;

  bool alloc(size_t nbytes, size_t* off) {
    std::lock_guard<std::mutex> g(mu);
    const size_t need = round_up(nbytes ? nbytes : 1, kPage);
    for (auto it = free_runs.begin(); it != free_runs.end(); ++it) {
      if (it->second >= need) {
        *off = it->first;
        const size_t rest = it->second - need;
        const size_t roff = it->first + need;
        free_runs.erase(it);
        if (rest) free_runs[roff] = rest;
        used += need;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t nbytes) {
    std::lock_guard<std::mutex> g(mu);
    const size_t len = round_up(nbytes ? nbytes : 1, kPage);
    used -= len;
    auto it = free_runs.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_runs.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_runs.erase(nx);
    }
    if (it != free_runs.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_runs.erase(it);
      }
    }
  }
};

namespace {

struct Logged {
  int basis = 0;  // 1: initial compression of |basis_index>
  unsigned long long basis_index = 0;
  std::vector<double> G;
  std::vector<int> targets, controls;
  unsigned int seq = 0;
  int in_id = 0, out_id = 1;
};

struct Region {
  size_t off = 0, bytes = 0;
  bool live = false;
  sv_pool* owner = nullptr;  // the pool the region lives in
};

}  // namespace

struct sv_state {
  sv_pool* pool = nullptr;
  int n = 0, sl = 0, b = 0, dtype = 2;
  double eb = 0.0;
  bool plain = false;
  QuantP qp{};
  double two2 = 0.0;
  cudaStream_t st = nullptr;
  // plain
  Region psi_r;
  void* psi = nullptr;
  // device copy of the current 4- or 5-qubit gate matrix (FP64, then its FP32 rounding),
  // written on the state's stream before each pass that uses it
  Region gate_r;  // plain states (compressed states keep it in their metadata run)
  double* gslot = nullptr;
  float* gslotf = nullptr;
  sv_pool* spill = nullptr;  // arenas and measurement buffers go here when `pool` is full
  // compressed
  unsigned long long nblocks = 0;
  Region meta_r, arena_r[2], aux_r;
  DevScalars* sc = nullptr;
  unsigned long long* toff[2] = {nullptr, nullptr};
  unsigned int* tlen[2] = {nullptr, nullptr};
  BlkInfo* binfo[2] = {nullptr, nullptr};
  double* vsum = nullptr;
  double* tree = nullptr;
  uint8_t* arena[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned int seq = 0;
  std::vector<Logged> log;
  // measurement scratch
  double* chunk[2] = {nullptr, nullptr};
  double* bins = nullptr;
  double* acc = nullptr;
  int* qdev = nullptr;
  unsigned long long chunk_amps = 0;
  int sticky_err = 0;
  // tracing: event pairs around the fused pass kernel
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free, ev_pending;
  double kernel_ms = 0.0;
  unsigned long long timed_passes = 0;
  unsigned long long io_base = 0;
  unsigned long long replayed = 0;  // passes re-run after an arena overflow
  int threads = 0;                  // CTA size of the fused pass (0: default)
  bool compact = false;             // register-capped build of the pass (1- and 2-qubit gates)
  int huff_chunk = 32;              // Huffman chunk size of the block format
  bool tensor_cores = true;         // 4- and 5-qubit complex128 gates on the tensor cores
  DevScalars* hsc = nullptr;        // pinned host copy of the device scalars
  bool hsc_valid = false;           // hsc holds the state after every submitted pass
  // passes between status checks (an overflow poisons every later pass until the check
  // replays them): about 2 ms of device work, 1 after an overflow
  int sync_every = 16;
  bool fixed_arena = false;  // the caller sized the arenas: they grow on overflow only
  std::chrono::steady_clock::time_point last_check = std::chrono::steady_clock::now();
  unsigned long long since_check = 0;  // passes submitted since the last clean check
};

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return SV_OK;
  std::fprintf(stderr, "libsv: CUDA error %s\n", cudaGetErrorString(e));
  return SV_ERR_CUDA;
}

uint8_t* pool_ptr(sv_pool* p, size_t off) { return p->base + off; }

bool region_alloc(sv_pool* p, Region* r, size_t bytes) {
  if (!p->alloc(bytes, &r->off)) return false;
  r->bytes = bytes;
  r->live = true;
  r->owner = p;
  return true;
}

void region_free(sv_pool* p, Region* r) {
  (void)p;
  if (r->live) r->owner->release(r->off, r->bytes);
  r->live = false;
}

uint8_t* region_ptr(const Region& r) { return r.owner->base + r.off; }

// A region of the state's pool, else of its spill pool.
bool region_alloc_spill(sv_state* s, Region* r, size_t bytes) {
  return region_alloc(s->pool, r, bytes) || (s->spill && region_alloc(s->spill, r, bytes));
}

int status_to_err(unsigned int st) {
  if (st & kStInternal) return SV_ERR_INTERNAL;
  if (st & kStCorrupt) return SV_ERR_CORRUPT;
  if (st & kStNorm) return SV_ERR_NORM;
  if (st & kStVerbatim) return SV_ERR_UNSUPPORTED;
  if (st & kStTimeout) return SV_ERR_TIMEOUT;
  if (st & kStOverflow) return SV_ERR_OOM;
  return SV_OK;
}

bool gate_args_ok(const sv_state* s, const int* targets, int k, const int* controls, int nc) {
  if (!targets || k < 1 || k > 5 || nc < 0 || (nc > 0 && !controls)) return false;
  unsigned long long seen = 0;
  for (int l = 0; l < k; ++l) {
    if (targets[l] < 0 || targets[l] >= s->n || ((seen >> targets[l]) & 1ull)) return false;
    seen |= 1ull << targets[l];
  }
  for (int l = 0; l < nc; ++l) {
    if (controls[l] < 0 || controls[l] >= s->n || ((seen >> controls[l]) & 1ull)) return false;
    seen |= 1ull << controls[l];
  }
  return true;
}

// The pass arguments of one logged step.
void build_args(const sv_state* s, const Logged& lg, PassArgs& a) {
  std::memset(&a, 0, sizeof(a));
  a.b = s->b;
  a.nv = 2 << s->b;
  a.qp = s->qp;
  a.two2 = s->two2;
  a.two_r = s->qp.two * s->qp.r;
  a.sc = s->sc;
  a.vsum = s->vsum;
  a.tree = s->tree;
  a.seq = lg.seq;
  a.in_arena = s->arena[lg.in_id];
  a.in_off = s->toff[lg.in_id];
  a.in_len = s->tlen[lg.in_id];
  a.out_arena = s->arena[lg.out_id];
  a.out_cap = s->arena_r[lg.out_id].bytes;
  a.out_id = lg.out_id;
  a.out_off = s->toff[lg.out_id];
  a.out_len = s->tlen[lg.out_id];
  a.threads = s->threads;
  a.chunk = s->huff_chunk;
  a.in_info = s->binfo[lg.in_id];
  a.out_info = s->binfo[lg.out_id];
  for (int g = 0; g < 4; ++g) a.pt_src[g] = -1;
  if (lg.basis) {
    a.input_basis = 1;
    a.basis = lg.basis_index;
    a.apply_gate = 0;
    a.use_sigma = 0;
    a.k = 0;
    a.K = 1;
    a.G = 1;
    a.h = 0;
    a.nlow = 0;
    a.pos_delta[0] = 0;
  } else {
    const int k = (int)lg.targets.size();
    a.k = k;
    a.K = 1 << k;
    a.apply_gate = 1;
    a.use_sigma = 1;
    int lows[5], nl = 0, highs[5], nh = 0;
    int hidx[5];
    for (int l = 0; l < k; ++l) {
      const int t = lg.targets[l];
      if (t < s->b) lows[nl++] = t;
      else {
        hidx[l] = nh;
        highs[nh++] = t - s->b;
      }
    }
    a.nlow = nl;
    a.h = nh;
    a.G = 1 << nh;
    std::vector<int> ls(lows, lows + nl), hs(highs, highs + nh);
    std::sort(ls.begin(), ls.end());
    std::sort(hs.begin(), hs.end());
    for (int l = 0; l < nl; ++l) a.low_t[l] = ls[l];
    for (int l = 0; l < nh; ++l) a.high_pos[l] = hs[l];
    for (int l = 0; l < nh; ++l) a.slot_shift[l] = highs[l];
    for (int m = 0; m < a.K; ++m) {
      int slot = 0, off = 0;
      for (int l = 0; l < k; ++l) {
        if (!((m >> l) & 1)) continue;
        const int t = lg.targets[l];
        if (t < s->b) off |= 1 << t;
        else slot |= 1 << hidx[l];
      }
      a.pos_delta[m] = slot * a.nv + 2 * off;
    }
    unsigned long long cm = 0;
    for (int c : lg.controls) cm |= 1ull << c;
    a.cmask = cm;
    if (a.K <= 8) {
      for (int e = 0; e < 2 * a.K * a.K; ++e) {
        a.g[e] = lg.G[e];
        a.gf[e] = (float)lg.G[e];
      }
    }
    a.gbig = s->gslot;
    a.gfbig = s->gslotf;
    // tensor cores for 4- and 5-qubit complex128 gates: 256-thread CTAs (the CTA size does not
    // change results), the stage holds the 128-tuple operand tile, and the CTA's shared memory
    // admits at most two CTAs per SM, whose tensor-memory columns then always fit
    if (s->tensor_cores && s->dtype == SV_C128 && a.K > 8 && threads_ok(s->b, 256) &&
        chunk_ok(s->b, s->huff_chunk, 256)) {
      const Layout Lb = make_layout(s->b, a.G, 8, false, true);
      if (Lb.stage_bytes >= (uint32_t)(kTcM * 2 * a.K * 2) && Lb.total + 1024 > 228u * 1024u / 3u) {
        a.tc = 1;
        a.threads = 256;
      }
    }
    // stream pass-through map: slot g keeps the codes of slot src when every row of the
    // members in g is a unit row (exactly 1) whose column is the same in-block position in
    // slot src; with in-block controls only src = g (the identity) qualifies
    a.cmask_high = cm & ~((1ull << s->b) - 1ull);
    const bool low_ctrl = (cm & ((1ull << s->b) - 1ull)) != 0;
    int mslot[32], moff[32];
    for (int m = 0; m < a.K; ++m) {
      mslot[m] = a.pos_delta[m] / a.nv;
      moff[m] = a.pos_delta[m] % a.nv;
    }
    int src[4] = {-2, -2, -2, -2};
    for (int jj = 0; jj < a.K; ++jj) {
      const int g = mslot[jj];
      int nz = 0, col = -1;
      a.need[g] |= 1u << g;
      for (int m = 0; m < a.K; ++m)
        if (lg.G[2 * (jj * a.K + m)] != 0.0 || lg.G[2 * (jj * a.K + m) + 1] != 0.0) {
          ++nz;
          col = m;
          a.need[g] |= 1u << mslot[m];
        }
      int sg = -1;
      if (nz == 1 && lg.G[2 * (jj * a.K + col)] == 1.0 && lg.G[2 * (jj * a.K + col) + 1] == 0.0 &&
          moff[col] == moff[jj])
        sg = mslot[col];
      if (low_ctrl && sg != g) sg = -1;
      src[g] = (src[g] == -2 || src[g] == sg) ? sg : -1;
    }
    for (int g = 0; g < a.G; ++g) a.pt_src[g] = src[g] < 0 ? -1 : src[g];
    a.pt_ok = s->dtype == SV_C128 ? 3 : 1;  // bit 0: zero blocks; bit 1: unit rows (complex128)
  }
  a.ngroups = s->nblocks >> a.h;
}

constexpr size_t kGateSlot = (size_t)2 * 32 * 32 * (sizeof(double) + sizeof(float));

// Copy a 4- or 5-qubit gate matrix to the state's device slot on its stream (the pass that
// reads it is launched after it on the same stream; the next copy waits for that pass).
cudaError_t upload_gate(const sv_state* s, const double* G, int K) {
  const size_t n = (size_t)2 * K * K;
  std::vector<float> gf(n);
  for (size_t e = 0; e < n; ++e) gf[e] = (float)G[e];
  // pageable sources: the calls return once the bytes are staged, so the buffers may go
  cudaError_t e = cudaMemcpyAsync(s->gslot, G, n * sizeof(double), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->gslotf, gf.data(), n * sizeof(float), cudaMemcpyHostToDevice, s->st);
  return e;
}

// Launch pass + norm tree + finalize for one logged step of one state.
int launch_logged(sv_state* s, const Logged& lg) {
  if (!s->arena[lg.in_id] || !s->arena[lg.out_id]) return SV_ERR_OOM;  // lost to a failed regrowth
  PassArgs a;
  build_args(s, lg, a);
  if (!lg.basis && a.K > 8) {
    const cudaError_t ge = upload_gate(s, lg.G.data(), a.K);
    if (ge != cudaSuccess) return cuda_err(ge);
  }
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (s->timing && !lg.basis) {
    if (s->ev_free.empty()) {
      cudaEventCreate(&ev.first);
      cudaEventCreate(&ev.second);
    } else {
      ev = s->ev_free.back();
      s->ev_free.pop_back();
    }
    cudaEventRecord(ev.first, s->st);
  }
  cudaError_t e = s->compact ? launch_pass_compact(a, s->dtype == SV_C64 ? 1 : 2, s->st)
                             : launch_pass(a, s->dtype == SV_C64 ? 1 : 2, s->st);
  if (e != cudaSuccess) return cuda_err(e);
  if (ev.first) {
    cudaEventRecord(ev.second, s->st);
    s->ev_pending.push_back(ev);
  }
  e = launch_norm(s->sc, s->vsum, s->nblocks, s->tree, s->two2, lg.out_id, lg.seq, s->st);
  return cuda_err(e);
}

// Record one step in a state's log (after its launch) and flip its arenas. Every 256 steps
// the state is checked (and an overflow replayed); an error that cannot be recovered (a
// collapsed norm, a corrupt stream) stays with the state — its own sv_sync reports it — and
// the state is no longer logged, so a batch carrying it goes on for the others.
int log_step(sv_state* s, Logged&& lg) {
  s->cur ^= 1;
  if (s->sticky_err) return SV_OK;
  s->log.push_back(std::move(lg));
  s->since_check++;
  s->hsc_valid = false;
  if (s->log.size() >= (size_t)s->sync_every) {
    const int rc = sv_sync(s);
    if (rc == SV_ERR_CUDA) return rc;
    if (rc) s->sticky_err = rc;
  }
  return SV_OK;
}

int submit(sv_state* s, Logged lg) {
  lg.seq = s->seq++;
  lg.in_id = s->cur;
  lg.out_id = s->cur ^ 1;
  int rc = launch_logged(s, lg);
  if (rc) return rc;
  rc = log_step(s, std::move(lg));
  return rc ? rc : s->sticky_err;
}

int read_scalars(sv_state* s, DevScalars* h) {
  DevScalars* dst = s->hsc ? s->hsc : h;  // pinned when available: one short transfer
  cudaError_t e = cudaMemcpyAsync(dst, s->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e == cudaSuccess && dst != h) *h = *dst;
  return cuda_err(e);
}

// The device scalars after every submitted pass: the copy the last clean sv_sync read, else a
// fresh read (callers have synchronized).
int current_scalars(sv_state* s, DevScalars* h) {
  if (s->hsc && s->hsc_valid) {
    *h = *s->hsc;
    return SV_OK;
  }
  return read_scalars(s, h);
}

// Give arena `id` (not the live one) at least `want` bytes when the pool has room; keeps
// the current size otherwise. Its content is not needed: the next pass overwrites it.
int reserve_arena(sv_state* s, int id, size_t want) {
  if (s->arena_r[id].bytes >= want) return SV_OK;
  const size_t old = s->arena_r[id].bytes;
  region_free(s->pool, &s->arena_r[id]);
  if (!region_alloc_spill(s, &s->arena_r[id], want) && !region_alloc_spill(s, &s->arena_r[id], old)) {
    s->arena[id] = nullptr;  // no arena: the state takes no more passes
    s->sticky_err = SV_ERR_OOM;
    return SV_ERR_OOM;
  }
  s->arena[id] = region_ptr(s->arena_r[id]);
  return SV_OK;
}

int grow_arena(sv_state* s, int id, size_t need) {
  // twice what the failed pass asked for: the passes after it (replayed next) tend to grow
  // further, and every overflow costs a replay
  size_t want = std::max(s->arena_r[id].bytes + s->arena_r[id].bytes / 2, 2 * need);
  region_free(s->pool, &s->arena_r[id]);
  if (!region_alloc_spill(s, &s->arena_r[id], want) && !region_alloc_spill(s, &s->arena_r[id], need)) {
    s->arena[id] = nullptr;  // no arena: the state takes no more passes
    s->sticky_err = SV_ERR_OOM;
    return SV_ERR_OOM;
  }
  s->arena[id] = region_ptr(s->arena_r[id]);
  return SV_OK;
}

int ensure_aux(sv_state* s) {
  if (s->aux_r.live) return SV_OK;
  const unsigned long long dim = 1ull << s->n;
  s->chunk_amps = std::min<unsigned long long>(dim, 1ull << 20);
  const size_t chunk_bytes = (size_t)s->chunk_amps * 16;
  const size_t bytes = 2 * chunk_bytes + (sizeof(double) << 16) + 64 + 4096;
  if (!region_alloc_spill(s, &s->aux_r, bytes)) return SV_ERR_OOM;
  uint8_t* p = region_ptr(s->aux_r);
  s->chunk[0] = (double*)p;
  s->chunk[1] = (double*)(p + chunk_bytes);
  s->bins = (double*)(p + 2 * chunk_bytes);
  s->acc = (double*)(p + 2 * chunk_bytes + (sizeof(double) << 16));
  s->qdev = (int*)(p + 2 * chunk_bytes + (sizeof(double) << 16) + 64);
  return SV_OK;
}

// Decoded FP64 amplitudes [start, start+count) (count <= chunk_amps) into dst (device), on
// stream `st` (the state's own stream unless a caller has ordered st after it).
int read_chunk(sv_state* s, unsigned long long start, unsigned long long count, double* dst,
               cudaStream_t st) {
  if (s->plain) return cuda_err(launch_plain_read(s->psi, s->dtype == SV_C64 ? 1 : 2, start, count, dst, st));
  const unsigned long long B = 1ull << s->b;
  const unsigned long long b0 = start / B, b1 = (start + count + B - 1) / B;
  // chunk sizes are multiples of B (start, count aligned by the callers)
  cudaError_t e = launch_read_blocks(s->arena[s->cur], s->toff[s->cur], s->tlen[s->cur], b0, b1 - b0,
                                     s->b, s->dtype == SV_C64 ? 1 : 2, s->qp, dst, s->sc, st);
  return cuda_err(e);
}
int read_chunk(sv_state* s, unsigned long long start, unsigned long long count, double* dst) {
  return read_chunk(s, start, count, dst, s->st);
}

int check_status(sv_state* s) {
  DevScalars h;
  int rc = read_scalars(s, &h);
  if (rc) return rc;
  return status_to_err(h.status);
}

}  // namespace

extern "C" {

const char* sv_version(void) { return "libsv 0.1 (sm_103a)"; }

int sv_pool_create(void* dev_base, size_t bytes, sv_pool** out) {
  if (!dev_base || !out || ((uintptr_t)dev_base & 255) || bytes < kPage) return SV_ERR_ARG;
  sv_pool* p = new sv_pool();
  p->base = (uint8_t*)dev_base;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, dev_base) == cudaSuccess && at.type == cudaMemoryTypeHost) {
    if (!at.devicePointer) {  // pinned but not mapped into the device's address space
      delete p;
      return SV_ERR_ARG;
    }
    p->host = true;
    p->base = (uint8_t*)at.devicePointer;
  } else {
    cudaGetLastError();
  }
  p->bytes = bytes / kPage * kPage;
  p->free_runs[0] = p->bytes;
  *out = p;
  return SV_OK;
}

int sv_pool_destroy(sv_pool* p) {
  if (!p) return SV_ERR_ARG;
  if (p->nstates || p->used) return SV_ERR_ARG;  // states (or spilled arenas) remain
  delete p;
  return SV_OK;
}

int sv_pool_usage(const sv_pool* p, size_t* used, size_t* cap) {
  if (!p) return SV_ERR_ARG;
  if (used) *used = p->used;
  if (cap) *cap = p->bytes;
  return SV_OK;
}

int sv_create_ex(sv_pool* pool, int n, int sl, int bl, double eb, int dtype, size_t arena_bytes,
                 void* stream, sv_state** out) {
  if (!pool || !out || n < 1 || n > 40 || (dtype != SV_C64 && dtype != SV_C128) || !(eb >= 0.0) ||
      !std::isfinite(eb))
    return SV_ERR_ARG;
  sv_state* s = new sv_state();
  s->pool = pool;
  s->n = n;
  s->dtype = dtype;
  s->eb = eb;
  s->st = (cudaStream_t)stream;
  s->plain = eb == 0.0;
  if (s->plain) {
    s->sl = sl;
    const size_t bytes = (size_t)(dtype == SV_C64 ? 8 : 16) << n;
    if (!region_alloc(pool, &s->psi_r, bytes)) {
      delete s;
      return SV_ERR_OOM;
    }
    s->psi = pool_ptr(pool, s->psi_r.off);
    if (!region_alloc(pool, &s->gate_r, kGateSlot)) {
      region_free(pool, &s->psi_r);
      delete s;
      return SV_ERR_OOM;
    }
    s->gslot = (double*)pool_ptr(pool, s->gate_r.off);
    s->gslotf = (float*)(s->gslot + 2 * 32 * 32);
    pool->nstates++;
    int rc = cuda_err(launch_plain_basis(s->psi, n, dtype == SV_C64 ? 1 : 2, 0, s->st));
    *out = s;
    return rc;
  }
  if (bl < 0) bl = std::min(sl, 12);
  if (bl < 5 || bl > 12 || bl > n || sl < bl || sl > n) {
    delete s;
    return SV_ERR_ARG;
  }
  s->sl = sl;
  s->b = bl;
  s->qp.eb = eb;
  s->qp.two = 2.0 * eb;
  s->qp.r = 1.0 / s->qp.two;
  s->two2 = s->qp.two * s->qp.two;
  s->nblocks = 1ull << (n - bl);
  // metadata run: scalars | tables 0, 1 | block summaries 0, 1 | vsum | tree scratch
  const size_t nb = s->nblocks;
  size_t off = 0;
  const size_t o_sc = off;
  off += round_up(sizeof(DevScalars), 256);
  const size_t o_off0 = off;
  off += round_up(nb * 8, 256);
  const size_t o_off1 = off;
  off += round_up(nb * 8, 256);
  const size_t o_len0 = off;
  off += round_up(nb * 4, 256);
  const size_t o_len1 = off;
  off += round_up(nb * 4, 256);
  const size_t o_info0 = off;
  off += round_up(nb * sizeof(BlkInfo), 256);
  const size_t o_info1 = off;
  off += round_up(nb * sizeof(BlkInfo), 256);
  const size_t o_vsum = off;
  off += round_up(nb * 8, 256);
  const size_t o_tree = off;
  off += round_up(2 * (nb / 256 + 1) * 8, 256);
  const size_t o_gate = off;
  off += round_up(kGateSlot, 256);
  if (!region_alloc(pool, &s->meta_r, off)) {
    delete s;
    return SV_ERR_OOM;
  }
  uint8_t* m = pool_ptr(pool, s->meta_r.off);
  s->sc = (DevScalars*)(m + o_sc);
  if (cudaHostAlloc((void**)&s->hsc, sizeof(DevScalars), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();  // pageable transfers instead
    s->hsc = nullptr;
  }
  s->toff[0] = (unsigned long long*)(m + o_off0);
  s->toff[1] = (unsigned long long*)(m + o_off1);
  s->tlen[0] = (unsigned int*)(m + o_len0);
  s->tlen[1] = (unsigned int*)(m + o_len1);
  s->binfo[0] = (BlkInfo*)(m + o_info0);
  s->binfo[1] = (BlkInfo*)(m + o_info1);
  s->vsum = (double*)(m + o_vsum);
  s->tree = (double*)(m + o_tree);
  s->gslot = (double*)(m + o_gate);
  s->gslotf = (float*)(s->gslot + 2 * 32 * 32);
  // arenas: the initial state is nearly all 16-byte CONST blocks
  const size_t init_cap = arena_bytes ? arena_bytes : std::max<size_t>(kPage, nb * 64);
  s->fixed_arena = arena_bytes != 0;
  for (int id = 0; id < 2; ++id) {
    if (!region_alloc(pool, &s->arena_r[id], init_cap)) {
      region_free(pool, &s->arena_r[0]);
      region_free(pool, &s->meta_r);
      if (s->hsc) cudaFreeHost(s->hsc);
      delete s;
      return SV_ERR_OOM;
    }
    s->arena[id] = region_ptr(s->arena_r[id]);
  }
  pool->nstates++;
  *out = s;
  return sv_reset_basis(s, 0);
}

int sv_create(sv_pool* pool, int n, int sl, double eb, int dtype, void* stream, sv_state** out) {
  return sv_create_ex(pool, n, sl, -1, eb, dtype, 0, stream, out);
}

int sv_destroy(sv_state* s) {
  if (!s) return SV_ERR_ARG;
  cudaStreamSynchronize(s->st);
  for (auto& ev : s->ev_free) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  for (auto& ev : s->ev_pending) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  if (s->hsc) cudaFreeHost(s->hsc);
  region_free(s->pool, &s->psi_r);
  region_free(s->pool, &s->gate_r);
  region_free(s->pool, &s->meta_r);
  region_free(s->pool, &s->arena_r[0]);
  region_free(s->pool, &s->arena_r[1]);
  region_free(s->pool, &s->aux_r);
  s->pool->nstates--;
  delete s;
  return SV_OK;
}

int sv_reset_basis(sv_state* s, uint64_t index) {
  if (!s || (index >> s->n)) return SV_ERR_ARG;
  if (s->plain) return cuda_err(launch_plain_basis(s->psi, s->n, s->dtype == SV_C64 ? 1 : 2, index, s->st));
  DevScalars h;
  std::memset(&h, 0, sizeof(h));
  h.fail_seq = 0xFFFFFFFFu;
  h.sigma = 1.0;
  h.norm = 1.0;
  cudaError_t e = cudaMemcpyAsync(s->sc, &h, sizeof(h), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);  // h is a stack buffer
  if (e != cudaSuccess) return cuda_err(e);
  s->log.clear();
  s->sticky_err = 0;
  Logged lg;
  lg.basis = 1;
  lg.basis_index = index;
  return submit(s, std::move(lg));
}

int sv_apply_gate(sv_state* s, const double* G, const int* targets, int k, const int* controls,
                  int nc) {
  if (!s || !G || !gate_args_ok(s, targets, k, controls, nc)) return SV_ERR_ARG;
  if (s->plain) {
    unsigned long long cm = 0;
    for (int l = 0; l < nc; ++l) cm |= 1ull << controls[l];
    if (k > 3) {
      const cudaError_t ge = upload_gate(s, G, 1 << k);
      if (ge != cudaSuccess) return cuda_err(ge);
    }
    return cuda_err(launch_plain_gate(s->psi, s->n, s->dtype == SV_C64 ? 1 : 2, G, targets, k, cm,
                                      s->gslot, s->st));
  }
  int nh = 0;
  for (int l = 0; l < k; ++l) nh += targets[l] >= s->b;
  if (nh > 2) return SV_ERR_UNSUPPORTED;
  // the CTA's shared memory must hold the group's blocks and, for 4- and 5-qubit gates, the
  // fixed-point matrix (4096-amplitude blocks with two high targets do not fit)
  if (make_layout(s->b, 1 << nh, s->dtype == SV_C64 ? 4 : 8, false, k > 3).total > 227u * 1024u)
    return SV_ERR_UNSUPPORTED;
  Logged lg;
  lg.G.assign(G, G + 2 * (1 << k) * (1 << k));
  lg.targets.assign(targets, targets + k);
  if (nc) lg.controls.assign(controls, controls + nc);
  return submit(s, std::move(lg));
}

int sv_sync(sv_state* s) {
  if (!s) return SV_ERR_ARG;
  if (s->plain) return cuda_err(cudaStreamSynchronize(s->st));
  for (int attempt = 0; attempt < 64; ++attempt) {
    DevScalars h;
    int rc = read_scalars(s, &h);
    if (rc) return rc;
    if (h.status == 0) {
      s->log.clear();
      s->hsc_valid = s->hsc != nullptr;
      // an overflow costs a replay of every pass since the failed one: check about every
      // 2 ms of device work (the passes since the last check, over the time they took), at
      // most 256 passes apart
      const auto now = std::chrono::steady_clock::now();
      if (s->since_check > 0) {
        const double per_pass =
            std::chrono::duration<double>(now - s->last_check).count() / (double)s->since_check;
        const double n = per_pass > 0.0 ? 2e-3 / per_pass : 256.0;
        s->sync_every = n >= 256.0 ? 256 : (n <= 1.0 ? 1 : (int)n);
      }
      s->last_check = now;
      s->since_check = 0;
      const size_t live = (size_t)h.bump[s->cur];
      // the arena the next pass writes gets room for twice the current state
      if (!s->fixed_arena) {
        rc = reserve_arena(s, s->cur ^ 1, 2 * live);
        if (rc) return rc;
      }
      for (auto& ev : s->ev_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.first, ev.second);
        s->kernel_ms += ms;
        s->timed_passes++;
        s->ev_free.push_back(ev);
      }
      s->ev_pending.clear();
      return SV_OK;
    }
    // a replay re-records its passes: drop the events of the failed attempt
    for (auto& ev : s->ev_pending) s->ev_free.push_back(ev);
    s->ev_pending.clear();
    if (h.status != kStOverflow) return status_to_err(h.status);
    s->sync_every = 1;
    // find the failed pass in the log
    size_t i = 0;
    while (i < s->log.size() && s->log[i].seq != h.fail_seq) ++i;
    if (i == s->log.size()) return SV_ERR_OOM;
    const Logged& f = s->log[i];
    rc = grow_arena(s, f.out_id, (size_t)h.bump[f.out_id]);
    if (rc) return rc;
    h.status = 0;
    h.fail_seq = 0xFFFFFFFFu;
    h.bump[f.out_id] = 0;
    std::memset(&h.acc, 0, sizeof(h.acc));
    cudaError_t e = cudaMemcpyAsync(s->sc, &h, sizeof(h), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_err(e);
    for (size_t j = i; j < s->log.size(); ++j) {
      rc = launch_logged(s, s->log[j]);
      if (rc) return rc;
      s->replayed++;
    }
  }
  return SV_ERR_OOM;
}

int sv_norm(sv_state* s, double* out) {
  if (!s || !out) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  if (s->plain) {
    // plain norm via a dot of the state with itself
    rc = ensure_aux(s);
    if (rc) return rc;
    cudaMemsetAsync(s->acc, 0, 4 * sizeof(double), s->st);
    const unsigned long long dim = 1ull << s->n;
    for (unsigned long long st = 0; st < dim; st += s->chunk_amps) {
      rc = read_chunk(s, st, s->chunk_amps, s->chunk[0]);
      if (rc) return rc;
      cudaError_t e = launch_dot_chunk(s->chunk[0], s->chunk[0], s->chunk_amps, s->acc, s->st);
      if (e != cudaSuccess) return cuda_err(e);
    }
    double h[4];
    cudaMemcpyAsync(h, s->acc, sizeof(h), cudaMemcpyDeviceToHost, s->st);
    cudaStreamSynchronize(s->st);
    *out = h[2];
    return SV_OK;
  }
  DevScalars h;
  rc = current_scalars(s, &h);
  if (rc) return rc;
  *out = h.norm;
  return SV_OK;
}

int sv_set_threads(sv_state* s, int threads) {
  if (!s || s->plain || (threads != 0 && !threads_ok(s->b, threads))) return SV_ERR_ARG;
  if (!chunk_ok(s->b, s->huff_chunk, threads ? threads : worker_threads(s->b))) return SV_ERR_ARG;
  s->threads = threads;
  return SV_OK;
}

int sv_set_chunk(sv_state* s, int chunk) {
  if (!s || s->plain) return SV_ERR_ARG;
  if (!chunk_ok(s->b, chunk, s->threads ? s->threads : worker_threads(s->b))) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  s->huff_chunk = chunk;
  return sv_reset_basis(s, 0);  // the stored streams were coded with the old chunk size
}

int sv_set_spill_pool(sv_state* s, sv_pool* spill) {
  if (!s || s->plain || spill == s->pool) return SV_ERR_ARG;
  s->spill = spill;
  return SV_OK;
}

int sv_set_tensor_cores(sv_state* s, int on) {
  if (!s || s->plain) return SV_ERR_ARG;
  s->tensor_cores = on != 0;
  return SV_OK;
}

int sv_set_compact(sv_state* s, int on) {
  if (!s || s->plain) return SV_ERR_ARG;
  s->compact = on != 0;
  return SV_OK;
}

int sv_stats(sv_state* s, sv_stats_t* out) {
  if (!s || !out) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  std::memset(out, 0, sizeof(*out));
  if (s->plain) {
    out->compressed_bytes = (uint64_t)(s->dtype == SV_C64 ? 8 : 16) << s->n;
    out->peak_compressed_bytes = out->compressed_bytes;
    return SV_OK;
  }
  DevScalars h;
  rc = current_scalars(s, &h);
  if (rc) return rc;
  out->pass_index = h.pass_index;
  out->compressed_bytes = h.last_bytes;
  out->table_bytes = s->nblocks * 12;
  out->n_blocks = s->nblocks;
  out->blocks_const = h.last.modes[0];
  out->blocks_huff = h.last.modes[1];
  out->blocks_pack = h.last.modes[2];
  out->n_verbatim = h.last.n_verbatim;
  out->n_escape = h.last.n_escape;
  out->norm = h.norm;
  out->sigma = h.sigma;
  out->blocks_reused = h.last.reused;
  out->replayed_passes = s->replayed;
  out->peak_compressed_bytes = h.peak_bytes;
  for (int id = 0; id < 2; ++id)
    if (s->arena_r[id].live && s->arena_r[id].owner != s->pool) out->spill_arena_bytes += s->arena_r[id].bytes;
  return SV_OK;
}

int sv_compressed_bytes(sv_state* s, uint64_t* out) {
  if (!s || !out) return SV_ERR_ARG;
  sv_stats_t st;
  int rc = sv_stats(s, &st);
  if (rc) return rc;
  *out = st.compressed_bytes;
  return SV_OK;
}

int sv_block_stream(sv_state* s, uint64_t b, uint8_t* out, size_t cap, size_t* len) {
  if (!s || s->plain || b >= s->nblocks || !len) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  unsigned long long off = 0;
  unsigned int l = 0;
  cudaMemcpyAsync(&off, s->toff[s->cur] + b, 8, cudaMemcpyDeviceToHost, s->st);
  cudaMemcpyAsync(&l, s->tlen[s->cur] + b, 4, cudaMemcpyDeviceToHost, s->st);
  cudaError_t e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return cuda_err(e);
  *len = l;
  if (!out) return SV_OK;
  if (cap < l) return SV_ERR_ARG;
  e = cudaMemcpy(out, s->arena[s->cur] + off, l, cudaMemcpyDefault);  // the arena may be host memory
  return cuda_err(e);
}

int sv_read_amplitudes(sv_state* s, uint64_t start, uint64_t count, double* out) {
  if (!s || !out || start + count > (1ull << s->n) || start + count < start) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  rc = ensure_aux(s);
  if (rc) return rc;
  const unsigned long long B = s->plain ? 1 : (1ull << s->b);
  unsigned long long pos = start;
  const unsigned long long end = start + count;
  while (pos < end) {
    const unsigned long long c0 = pos / B * B;  // aligned chunk start
    unsigned long long c1 = std::min<unsigned long long>(c0 + s->chunk_amps, 1ull << s->n);
    rc = read_chunk(s, c0, c1 - c0, s->chunk[0]);
    if (rc) return rc;
    const unsigned long long take = std::min(c1, end) - pos;
    cudaError_t e = cudaMemcpyAsync(out + 2 * (pos - start), s->chunk[0] + 2 * (pos - c0), take * 16,
                                    cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_err(e);
    pos += take;
  }
  return s->plain ? SV_OK : check_status(s);
}

int sv_amplitudes(sv_state* s, const uint64_t* idx, size_t cnt, double* out) {
  if (!s || (cnt && (!idx || !out))) return SV_ERR_ARG;
  for (size_t i = 0; i < cnt; ++i) {
    int rc = sv_read_amplitudes(s, idx[i], 1, out + 2 * i);
    if (rc) return rc;
  }
  return SV_OK;
}

int sv_measure_probs(sv_state* s, const int* qubits, int m, double* out) {
  if (!s || !qubits || !out || m < 1 || m > 14) return SV_ERR_ARG;
  for (int l = 0; l < m; ++l)
    if (qubits[l] < 0 || qubits[l] >= s->n) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  rc = ensure_aux(s);
  if (rc) return rc;
  cudaMemsetAsync(s->bins, 0, sizeof(double) << m, s->st);
  int qh[16];
  for (int l = 0; l < m; ++l) qh[l] = qubits[l];
  cudaMemcpyAsync(s->qdev, qh, sizeof(int) * m, cudaMemcpyHostToDevice, s->st);
  const unsigned long long dim = 1ull << s->n;
  for (unsigned long long st = 0; st < dim; st += s->chunk_amps) {
    rc = read_chunk(s, st, s->chunk_amps, s->chunk[0]);
    if (rc) return rc;
    cudaError_t e = launch_probs_chunk(s->chunk[0], st, s->chunk_amps, s->qdev, m, s->bins, s->st);
    if (e != cudaSuccess) return cuda_err(e);
  }
  std::vector<double> h((size_t)1 << m);
  cudaError_t e = cudaMemcpyAsync(h.data(), s->bins, sizeof(double) << m, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return cuda_err(e);
  double tot = 0.0;
  for (double v : h) tot += v;
  if (!(tot > 0.0)) return SV_ERR_NORM;
  for (size_t i = 0; i < h.size(); ++i) out[i] = h[i] / tot;
  return s->plain ? SV_OK : check_status(s);
}

int sv_fidelity(sv_state* a, sv_state* b, double* out) {
  if (!a || !b || !out || a->n != b->n) return SV_ERR_ARG;
  int rc = sv_sync(a);
  if (!rc && b != a) rc = sv_sync(b);
  if (rc) return rc;
  rc = ensure_aux(a);
  if (!rc) rc = ensure_aux(b);
  if (rc) return rc;
  // work on a's stream: b's blocks are read there too, after an event that orders a's stream
  // behind everything submitted on b's (b itself is not modified)
  if (b->st != a->st) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, b->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(a->st, ev, 0);
    if (ev) cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_err(e);
  }
  const unsigned long long dim = 1ull << a->n;
  const unsigned long long ch = std::min(a->chunk_amps, b->chunk_amps);
  cudaMemsetAsync(a->acc, 0, 4 * sizeof(double), a->st);
  for (unsigned long long st = 0; st < dim; st += ch) {
    rc = read_chunk(a, st, ch, a->chunk[0]);
    if (rc) return rc;
    rc = read_chunk(b, st, ch, a->chunk[1], a->st);
    if (rc) return rc;
    cudaError_t e = launch_dot_chunk(a->chunk[0], a->chunk[1], ch, a->acc, a->st);
    if (e != cudaSuccess) return cuda_err(e);
  }
  double h[4];
  cudaError_t e = cudaMemcpyAsync(h, a->acc, sizeof(h), cudaMemcpyDeviceToHost, a->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->st);
  if (e != cudaSuccess) return cuda_err(e);
  if (!(h[2] > 0.0) || !(h[3] > 0.0)) return SV_ERR_NORM;
  *out = (h[0] * h[0] + h[1] * h[1]) / (h[2] * h[3]);
  if (!a->plain && (rc = check_status(a))) return rc;
  if (!b->plain && (rc = check_status(b))) return rc;
  return SV_OK;
}

int sv_set_pass_timing(sv_state* s, int on) {
  if (!s || s->plain) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  DevScalars h;
  rc = read_scalars(s, &h);
  if (rc) return rc;
  s->timing = on != 0;
  s->kernel_ms = 0.0;
  s->timed_passes = 0;
  s->io_base = h.io_bytes;
  return SV_OK;
}

int sv_get_pass_timing(sv_state* s, double* kernel_ms, uint64_t* passes, uint64_t* bytes) {
  if (!s || s->plain) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  DevScalars h;
  rc = read_scalars(s, &h);
  if (rc) return rc;
  if (kernel_ms) *kernel_ms = s->kernel_ms;
  if (passes) *passes = s->timed_passes;
  // per block: offset + length read (12) and written (12), summary read and written (32),
  // verbatim sum written (8)
  if (bytes) *bytes = (h.io_bytes - s->io_base) + 64ull * s->nblocks * s->timed_passes;
  return SV_OK;
}

}  // extern "C"

namespace {

constexpr int kRing = 4;

struct GraphKey {
  int count, kmax, gmax;
  unsigned long long groups;
  bool operator<(const GraphKey& o) const {
    if (count != o.count) return count < o.count;
    if (kmax != o.kmax) return kmax < o.kmax;
    if (gmax != o.gmax) return gmax < o.gmax;
    return groups < o.groups;
  }
};

}  // namespace

struct sv_batch {
  sv_pool* pool = nullptr;
  cudaStream_t st = nullptr;
  int max_states = 0;
  Region dev_r;
  uint8_t* d_blob = nullptr;
  size_t blob_bytes = 0;
  size_t off_prefix = 0;
  uint8_t* h_buf[kRing] = {nullptr};
  cudaEvent_t h_done[kRing] = {nullptr};
  int ring = 0;
  bool graphs = false;
  std::map<GraphKey, std::vector<cudaGraphExec_t>> cache;
  std::map<GraphKey, int> seen;  // shapes run once uncaptured (their kernels are set up)
  unsigned long long steps = 0;
};

extern "C" {

int sv_batch_create(sv_pool* pool, int max_states, void* stream, sv_batch** out) {
  if (!pool || !out || max_states < 1 || max_states > 65536) return SV_ERR_ARG;
  sv_batch* bt = new sv_batch();
  bt->pool = pool;
  bt->st = (cudaStream_t)stream;
  bt->max_states = max_states;
  size_t off = (size_t)max_states * sizeof(PassArgs);
  bt->off_prefix = off;
  off += round_up((size_t)(max_states + 1) * 8, 256);
  bt->blob_bytes = off;
  if (!region_alloc(pool, &bt->dev_r, off)) {
    delete bt;
    return SV_ERR_OOM;
  }
  bt->d_blob = pool_ptr(pool, bt->dev_r.off);
  for (int r = 0; r < kRing; ++r) {
    if (cudaHostAlloc((void**)&bt->h_buf[r], off, cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->h_done[r], cudaEventDisableTiming) != cudaSuccess) {
      sv_batch_destroy(bt);
      return SV_ERR_CUDA;
    }
  }
  pool->nstates++;
  *out = bt;
  return SV_OK;
}

int sv_batch_destroy(sv_batch* bt) {
  if (!bt) return SV_ERR_ARG;
  cudaStreamSynchronize(bt->st);
  for (auto& kv : bt->cache)
    for (auto g : kv.second) cudaGraphExecDestroy(g);
  for (int r = 0; r < kRing; ++r) {
    if (bt->h_buf[r]) cudaFreeHost(bt->h_buf[r]);
    if (bt->h_done[r]) cudaEventDestroy(bt->h_done[r]);
  }
  if (bt->dev_r.live) {
    region_free(bt->pool, &bt->dev_r);
    bt->pool->nstates--;
  }
  delete bt;
  return SV_OK;
}

int sv_batch_ready(sv_batch* bt) {
  if (!bt) return SV_ERR_ARG;
  const cudaError_t e = cudaEventQuery(bt->h_done[bt->ring]);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return cuda_err(e);
}

int sv_batch_use_graphs(sv_batch* bt, int on) {
  if (!bt) return SV_ERR_ARG;
  bt->graphs = on != 0;
  return SV_OK;
}

int sv_batch_apply(sv_batch* bt, sv_state* const* states, const sv_gate_t* gates, int count) {
  if (!bt || !states || !gates || count < 1 || count > bt->max_states) return SV_ERR_ARG;
  const sv_state* s0 = states[0];
  if (!s0) return SV_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    const sv_state* s = states[i];
    const sv_gate_t& g = gates[i];
    if (!s || s->plain || s->dtype != s0->dtype || s->b != s0->b || s->huff_chunk != s0->huff_chunk || s->st != bt->st || !g.G ||
        !gate_args_ok(s, g.targets, g.k, g.controls, g.n_controls))
      return SV_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (states[j] == s) return SV_ERR_ARG;  // one gate per state per step
    int nh = 0;
    for (int l = 0; l < g.k; ++l) nh += g.targets[l] >= s->b;
    if (nh > 2 || g.k > 3) return SV_ERR_UNSUPPORTED;  // batches: gates of at most 3 qubits
    if (!s->arena[0] || !s->arena[1]) return SV_ERR_OOM;  // lost to a failed regrowth
  }
  // stage descriptors and tables in the next pinned buffer of the ring
  const int slot = bt->ring;
  bt->ring = (bt->ring + 1) % kRing;
  cudaError_t e = cudaEventSynchronize(bt->h_done[slot]);  // its previous copy has run
  if (e != cudaSuccess) return cuda_err(e);
  uint8_t* hb = bt->h_buf[slot];
  PassArgs* hd = (PassArgs*)hb;
  unsigned long long* hp = (unsigned long long*)(hb + bt->off_prefix);
  std::vector<Logged> logs((size_t)count);
  int kmax = 1, gmax = 1;
  hp[0] = 0;
  for (int i = 0; i < count; ++i) {
    sv_state* s = states[i];
    const sv_gate_t& g = gates[i];
    Logged& lg = logs[(size_t)i];
    lg.G.assign(g.G, g.G + 2 * (1 << g.k) * (1 << g.k));
    lg.targets.assign(g.targets, g.targets + g.k);
    if (g.n_controls) lg.controls.assign(g.controls, g.controls + g.n_controls);
    lg.seq = s->seq++;
    lg.in_id = s->cur;
    lg.out_id = s->cur ^ 1;
    build_args(s, lg, hd[i]);
    hp[i + 1] = hp[i] + hd[i].ngroups;
    kmax = std::max(kmax, hd[i].K);
    gmax = std::max(gmax, hd[i].G);
  }
  const int kbucket = kmax <= 2 ? 2 : (kmax <= 4 ? 4 : 8);
  const PassArgs* d_descs = (const PassArgs*)bt->d_blob;
  const unsigned long long* d_prefix = (const unsigned long long*)(bt->d_blob + bt->off_prefix);
  auto enqueue = [&](uint8_t* src) -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(bt->d_blob, src, bt->blob_bytes, cudaMemcpyHostToDevice, bt->st);
    if (r == cudaSuccess)
      r = launch_pass_batch(d_descs, d_prefix, count, hp[count], s0->b, gmax, kbucket,
                            s0->dtype == SV_C64 ? 1 : 2, s0->threads, s0->huff_chunk, bt->st);
    if (r == cudaSuccess) r = launch_norm_batch(d_descs, count, bt->st);
    return r;
  };
  GraphKey key{count, kbucket, gmax, hp[count]};
  auto it = bt->cache.find(key);
  const bool seen_before = bt->seen[key]++ > 0;
  if (bt->graphs && it == bt->cache.end() && seen_before) {
    // capture one graph per ring slot (each copies from its own pinned buffer)
    std::vector<cudaGraphExec_t> execs;
    for (int r = 0; r < kRing && e == cudaSuccess; ++r) {
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(bt->st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = enqueue(bt->h_buf[r]);
        e = cudaStreamEndCapture(bt->st, &graph);
        if (e == cudaSuccess) e = e2;
      }
      cudaGraphExec_t ex = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e == cudaSuccess) execs.push_back(ex);
    }
    if (e != cudaSuccess) return cuda_err(e);
    it = bt->cache.emplace(key, std::move(execs)).first;
  }
  if (bt->graphs && it != bt->cache.end()) e = cudaGraphLaunch(it->second[(size_t)slot], bt->st);
  else e = enqueue(hb);
  if (e == cudaSuccess) e = cudaEventRecord(bt->h_done[slot], bt->st);
  if (e != cudaSuccess) return cuda_err(e);
  bt->steps++;
  int rc = SV_OK;
  for (int i = 0; i < count; ++i) {
    const int r = log_step(states[i], std::move(logs[(size_t)i]));
    if (r && !rc) rc = r;
  }
  return rc;
}

int sv_overlap_qft(sv_state* s, uint64_t x, double* out) {
  if (!s || !out || (x >> s->n) || s->n < 1) return SV_ERR_ARG;
  int rc = sv_sync(s);
  if (rc) return rc;
  rc = ensure_aux(s);
  if (rc) return rc;
  cudaMemsetAsync(s->acc, 0, 4 * sizeof(double), s->st);
  const unsigned long long dim = 1ull << s->n;
  for (unsigned long long st = 0; st < dim; st += s->chunk_amps) {
    rc = read_chunk(s, st, s->chunk_amps, s->chunk[0]);
    if (rc) return rc;
    cudaError_t e = launch_qft_overlap_chunk(s->chunk[0], st, s->chunk_amps, x, s->n, s->acc, s->st);
    if (e != cudaSuccess) return cuda_err(e);
  }
  double h[4];
  cudaError_t e = cudaMemcpyAsync(h, s->acc, sizeof(h), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return cuda_err(e);
  const double scale = 1.0 / std::sqrt(std::ldexp(1.0, s->n));  // 2^{-n/2}
  out[0] = h[0] * scale;
  out[1] = h[1] * scale;
  out[2] = h[2];
  return s->plain ? SV_OK : check_status(s);
}

size_t sv_codec_scratch_bytes(void) { return round_up(sizeof(DevScalars), 256); }

int sv_codec_compress(const void* values, uint64_t nblocks, int bl, int dtype, double eb, void* out,
                      uint64_t cap, uint64_t* offsets, uint32_t* lengths, void* scratch,
                      void* stream, uint64_t* used) {
  if (bl < 5 || bl > 12 || (dtype != SV_C64 && dtype != SV_C128) || !(eb > 0.0) || !std::isfinite(eb))
    return SV_ERR_ARG;
  if (nblocks == 0) {  // nothing to compress (the buffers may be NULL)
    if (used) *used = 0;
    return SV_OK;
  }
  if (!values || !out || !offsets || !lengths || !scratch || ((uintptr_t)out & 15) || ((uintptr_t)scratch & 15))
    return SV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  DevScalars* sc = (DevScalars*)scratch;
  QuantP qp;
  qp.eb = eb;
  qp.two = 2.0 * eb;
  qp.r = 1.0 / qp.two;
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st);
  if (e != cudaSuccess) return cuda_err(e);
  e = launch_codec_compress(values, nblocks, bl, dtype == SV_C64 ? 1 : 2, qp, (uint8_t*)out, cap,
                            (unsigned long long*)offsets, lengths, sc, nullptr, st);
  if (e != cudaSuccess) return cuda_err(e);
  DevScalars h;
  e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e);
  if (used) *used = h.bump[0];
  return status_to_err(h.status);
}

int sv_codec_decompress(const void* in, const uint64_t* offsets, const uint32_t* lengths,
                        uint64_t nblocks, int bl, int dtype, double eb, void* values, void* scratch,
                        void* stream) {
  if (bl < 5 || bl > 12 || (dtype != SV_C64 && dtype != SV_C128) || !(eb > 0.0) || !std::isfinite(eb))
    return SV_ERR_ARG;
  if (nblocks == 0) return SV_OK;  // nothing to decode (the buffers may be NULL)
  if (!in || !offsets || !lengths || !values || !scratch || ((uintptr_t)in & 15) || ((uintptr_t)scratch & 15))
    return SV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  DevScalars* sc = (DevScalars*)scratch;
  QuantP qp;
  qp.eb = eb;
  qp.two = 2.0 * eb;
  qp.r = 1.0 / qp.two;
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st);
  if (e != cudaSuccess) return cuda_err(e);
  e = launch_codec_decompress((const uint8_t*)in, (const unsigned long long*)offsets, lengths, nblocks,
                              bl, dtype == SV_C64 ? 1 : 2, qp, values, sc, st);
  if (e != cudaSuccess) return cuda_err(e);
  DevScalars h;
  e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e);
  return status_to_err(h.status);
}

}  // extern "C"
