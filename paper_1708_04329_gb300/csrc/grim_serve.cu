// grim_server: continuous batching of filter requests over a resident index.
//
// The index stays in device memory for the server's life.  Requests (read
// batches of any size, lengths and edit budgets, with or without candidate
// lists) are copied at submission into a host-side queue.  One scheduler
// thread owns S slots, each a host-memory plan (grim_plan with
// GRIM_PLAN_HOST_IO) with its own stream: whenever a slot is free it merges
// the queued requests, oldest first, into one batch up to the slot's read,
// byte and candidate limits, writes them into the slot's mapped input
// buffers and launches the slot's graph.  Requests that arrive while other
// batches run are admitted as slots free up, and the batches of different
// slots run concurrently on the device.  S is bounded by a device-memory
// budget for the slots' batch buffers, workspaces and pass lists.
//
// With max_chunk_reads set, a request is queued as chunks of consecutive
// reads (at most that many reads, and within the slot's byte and candidate
// limits), which may run in different slots and batches; the request
// completes when its last chunk does, with the chunks' records joined in
// read order.  A request larger than one slot is then accepted too.
//
// A merged batch's pass list is sorted by batch-local read, so each chunk's
// records are one contiguous run; they are handed back with the request's
// own read numbering.  The filter's arithmetic is per read, so a request's
// result does not depend on what it was merged with or how it was cut.  A
// batch whose pass list overflows the slot's capacity is split: its chunks
// go back to the head of the queue to be run one per batch, and a single
// chunk that still overflows completes its request with GRIM_E_OVERFLOW and
// the request's total.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "grim.h"

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request;

// A run of consecutive reads of a request that is queued, batched and run as
// one unit: the whole request, or one chunk of a split request.
struct Piece {
  Request* req = nullptr;
  uint32_t read0 = 0, n_reads = 0;  // reads [read0, read0 + n_reads) of the request
  uint64_t byte0 = 0, n_bases = 0;  // their bytes: request reads[byte0, byte0 + n_bases)
  uint64_t cand0 = 0, n_cand = 0;   // their candidates: request cand[cand0, cand0 + n_cand)
  bool solo = false;                // run alone (its merged batch overflowed)
  bool started = false;             // handed to a slot at least once
  int status = GRIM_OK;
  uint64_t n_out = 0;
  std::vector<uint32_t> out_read, out_bin;  // request-local read numbers
  std::vector<uint8_t> out_count;
};

struct Request {
  uint64_t ticket = 0;
  uint32_t n_reads = 0;
  std::vector<char> reads;
  std::vector<uint64_t> offsets;
  std::vector<uint32_t> lens;
  std::vector<uint16_t> e;
  std::vector<int32_t> cand;
  std::vector<uint64_t> cand_off;
  std::vector<Piece> pieces;  // fixed after submission (queued by address)
  uint32_t pieces_left = 0;   // pieces not yet completed
  bool done = false;
  int status = GRIM_OK;
  uint64_t n_out = 0;
  std::vector<uint32_t> out_read, out_bin;
  std::vector<uint8_t> out_count;
  grim_request_info info{};

  void release_inputs() {
    reads = {};
    offsets = {};
    lens = {};
    e = {};
    cand = {};
    cand_off = {};
  }
};

struct Slot {
  grim_plan* plan = nullptr;
  grim_plan_buffers buf{};
  cudaStream_t stream = nullptr;
  bool busy = false;
  uint64_t batch = 0;
  std::vector<Piece*> pieces;
  std::vector<uint32_t> first_read;  // batch-local read number of each piece's first read
};

}  // namespace

struct grim_server {
  const grim_index* idx = nullptr;
  grim_server_desc d{};
  grim_index_desc ix{};
  bool cand_mode = false;
  int device = 0;
  std::vector<Slot> slots;
  uint64_t device_bytes = 0;

  std::mutex mu;
  std::condition_variable cv_work;  // scheduler: something was queued, or stop
  std::condition_variable cv_done;  // waiters: a request completed
  std::deque<Piece*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  uint64_t queued_reads = 0;
  grim_server_stats st{};
  bool stop = false;
  int fatal = GRIM_OK;  // a CUDA failure that ended the scheduler
  std::thread worker;

  // ---- scheduler side (worker thread only, except where the lock is taken)

  // Merge queued requests into slot s; returns false if the queue was
  // empty.  Called with the lock held.
  bool form(Slot& s) {
    if (queue.empty()) return false;
    s.pieces.clear();
    s.first_read.clear();
    uint32_t nr = 0;
    uint64_t nb = 0, nc = 0;
    while (!queue.empty()) {
      Piece* p = queue.front();
      const bool first = s.pieces.empty();
      if (!first && (p->solo || s.pieces.front()->solo)) break;
      if (!first && ((uint64_t)nr + p->n_reads > d.max_reads || nb + p->n_bases > d.max_bases ||
                     nc + p->n_cand > d.max_cand))
        break;
      queue.pop_front();
      queued_reads -= p->n_reads;
      p->started = true;
      s.pieces.push_back(p);
      s.first_read.push_back(nr);
      nr += p->n_reads;
      nb += p->n_bases;
      nc += p->n_cand;
    }
    s.batch = ++st.batches;
    st.batch_reads += nr;
    return true;
  }

  // Copy the slot's requests into its mapped inputs and launch (no lock).
  int launch(Slot& s) {
    const uint64_t t = now_ns();
    uint64_t nb = 0, nc = 0;
    uint32_t nr = 0;
    for (Piece* p : s.pieces) {
      const Request* r = p->req;
      if (p->n_bases) std::memcpy(s.buf.reads + nb, r->reads.data() + p->byte0, p->n_bases);
      for (uint32_t i = 0; i < p->n_reads; ++i) {
        const uint32_t k = p->read0 + i;
        s.buf.offsets[nr + i] = nb + (r->offsets[k] - p->byte0);
        s.buf.lens[nr + i] = r->lens[k];
        s.buf.e[nr + i] = r->e[k];
      }
      if (cand_mode) {
        if (p->n_cand)
          std::memcpy(s.buf.cand + nc, r->cand.data() + p->cand0, p->n_cand * sizeof(int32_t));
        for (uint32_t i = 0; i < p->n_reads; ++i)
          s.buf.cand_off[nr + i] = nc + (r->cand_off[p->read0 + i] - p->cand0);
      }
      if (!p->req->info.t_launch_ns) p->req->info.t_launch_ns = t;
      nb += p->n_bases;
      nc += p->n_cand;
      nr += p->n_reads;
    }
    if (cand_mode) s.buf.cand_off[nr] = nc;
    const int rc = grim_plan_launch(s.plan, nr, nc, s.stream);
    s.busy = rc == GRIM_OK;
    return rc;
  }

  // The slot's batch has finished: hand each piece its records, and complete
  // the requests whose last piece this was.  Called with the lock held.
  void finish(Slot& s, int rc, uint64_t n_out) {
    const uint32_t npc = (uint32_t)s.pieces.size();
    uint32_t batch_reads = 0;
    for (Piece* p : s.pieces) batch_reads += p->n_reads;
    if (rc == GRIM_E_OVERFLOW && npc > 1) {
      // run the pieces again, one batch each, in their order
      for (uint32_t i = npc; i-- > 0;) {
        Piece* p = s.pieces[i];
        p->solo = true;
        queue.push_front(p);
        queued_reads += p->n_reads;
      }
      st.overflow_splits++;
      s.pieces.clear();
      return;
    }
    if (rc == GRIM_OK) {
      // records are sorted by batch-local read: walk the pieces alongside
      uint32_t k = 0;
      std::vector<uint64_t> begin(npc + 1, n_out);
      for (uint64_t i = 0; i < n_out; ++i) {
        const uint32_t rd = s.buf.out_read[i];
        while (k < npc && rd >= s.first_read[k]) begin[k++] = i;
      }
      for (uint32_t j = 0; j < npc; ++j) {
        Piece* p = s.pieces[j];
        const uint64_t a = begin[j], b = begin[j + 1];
        const uint32_t shift = p->read0 - s.first_read[j];  // batch-local -> request-local
        p->n_out = b - a;
        p->out_read.resize(b - a);
        p->out_bin.assign(s.buf.out_bin + a, s.buf.out_bin + b);
        p->out_count.assign(s.buf.out_count + a, s.buf.out_count + b);
        for (uint64_t i = a; i < b; ++i) p->out_read[i - a] = s.buf.out_read[i] + shift;
      }
    }
    const uint64_t t = now_ns();
    for (Piece* p : s.pieces) {
      p->status = rc;
      if (rc == GRIM_E_OVERFLOW) p->n_out = n_out;
      Request* r = p->req;
      r->info.batch = s.batch;
      r->info.batch_requests = npc;
      r->info.batch_reads = batch_reads;
      if (--r->pieces_left == 0) complete(r, t);
    }
    s.pieces.clear();
    cv_done.notify_all();
  }

  // All of a request's pieces have run: join their records in read order.
  void complete(Request* r, uint64_t t) {
    r->status = GRIM_OK;
    r->n_out = 0;
    for (const Piece& p : r->pieces) {
      if (p.status != GRIM_OK && r->status == GRIM_OK) r->status = p.status;
      r->n_out += p.n_out;
    }
    if (r->status == GRIM_OK) {
      r->out_read.reserve(r->n_out);
      r->out_bin.reserve(r->n_out);
      r->out_count.reserve(r->n_out);
      for (Piece& p : r->pieces) {
        r->out_read.insert(r->out_read.end(), p.out_read.begin(), p.out_read.end());
        r->out_bin.insert(r->out_bin.end(), p.out_bin.begin(), p.out_bin.end());
        r->out_count.insert(r->out_count.end(), p.out_count.begin(), p.out_count.end());
        p.out_read = {};
        p.out_bin = {};
        p.out_count = {};
      }
    }
    r->done = true;
    r->info.status = r->status;
    r->info.n_out = r->n_out;
    r->info.t_done_ns = t;
    r->release_inputs();
    st.completed++;
    st.reads_done += r->n_reads;
    st.records += r->n_out;
  }

  void fail_all(int rc) {
    std::lock_guard<std::mutex> g(mu);
    fatal = rc;
    auto fail = [&](Piece* p) {
      Request* r = p->req;
      if (r->done) return;
      r->status = rc;
      r->done = true;
      r->info.status = rc;
      r->info.t_done_ns = now_ns();
    };
    for (Slot& s : slots) {
      for (Piece* p : s.pieces) fail(p);
      s.pieces.clear();
      s.busy = false;
    }
    for (Piece* p : queue) fail(p);
    queue.clear();
    queued_reads = 0;
    cv_done.notify_all();
  }

  // the scheduler thread: any exception (an allocation failing while a
  // result is copied) ends the server with GRIM_E_NOMEM rather than the process
  void run() {
    try {
      loop();
    } catch (...) {
      fail_all(GRIM_E_NOMEM);
    }
  }

  void loop() {
    cudaSetDevice(device);
    uint32_t idle_spins = 0;
    for (;;) {
      bool progress = false;
      // 1. collect finished batches
      for (Slot& s : slots) {
        if (!s.busy) continue;
        const int q = grim_plan_query(s.plan);
        if (q == GRIM_E_NOT_READY) continue;
        uint64_t n_out = 0;
        const int rc = q == GRIM_OK ? grim_plan_wait(s.plan, &n_out) : q;
        s.busy = false;
        if (rc == GRIM_E_CUDA) {
          fail_all(rc);
          return;
        }
        std::lock_guard<std::mutex> g(mu);
        finish(s, rc, n_out);
        progress = true;
      }
      // 2. fill free slots from the queue
      for (Slot& s : slots) {
        if (s.busy) continue;
        {
          std::lock_guard<std::mutex> g(mu);
          if (!form(s)) break;
        }
        const int rc = launch(s);
        if (rc != GRIM_OK) {
          fail_all(rc);
          return;
        }
        progress = true;
      }
      bool any_busy = false;
      for (const Slot& s : slots) any_busy |= s.busy;
      if (progress) {
        idle_spins = 0;
        continue;
      }
      if (any_busy) {
        // a batch is on the device: poll its event (short naps after a while)
        if (++idle_spins < 2000) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(20));
        continue;
      }
      // nothing on the device: sleep until a request arrives or the server stops
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      if (stop && queue.empty()) return;
      idle_spins = 0;
    }
  }
};

namespace {

void destroy_slots(grim_server* s) {
  for (Slot& sl : s->slots) {
    if (sl.plan) grim_plan_free(sl.plan);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  s->slots.clear();
}

// Check one request against the server's limits and the index, so that a
// merged batch cannot fail because of one of its members, and cut it into
// pieces: the whole request, or (max_chunk_reads set) chunks of consecutive
// reads, each within max_chunk_reads reads and the slot's byte and
// candidate limits.
int validate(const grim_server* s, const char* reads, const uint64_t* offsets,
             const uint32_t* lens, uint32_t n_reads, const uint16_t* e, const int32_t* cand,
             const uint64_t* cand_off, std::vector<Piece>* pieces) {
  if (n_reads && (!reads || !offsets || !lens || !e)) return GRIM_E_ARG;
  const uint32_t chunk = s->d.max_chunk_reads;
  if (!chunk && n_reads > s->d.max_reads) return GRIM_E_ARG;
  for (uint32_t i = 0; i < n_reads; ++i) {
    const uint64_t l = lens[i];
    if (l < s->ix.q) return GRIM_E_READ_TOO_SHORT;
    if (l > s->ix.max_read_len || l - s->ix.q + 1 > 255) return GRIM_E_READ_TOO_LONG;
    if (e[i] > s->d.max_e) return GRIM_E_ARG;
    if (offsets[i] > UINT64_MAX - l || l > s->d.max_bases) return GRIM_E_ARG;
    if (!chunk && offsets[i] + l > s->d.max_bases) return GRIM_E_ARG;
  }
  if (s->cand_mode) {
    if (!cand_off) return GRIM_E_ARG;
    if (cand_off[0] != 0) return GRIM_E_ARG;
    for (uint32_t i = 0; i < n_reads; ++i) {
      if (cand_off[i + 1] < cand_off[i]) return GRIM_E_ARG;
      if (cand_off[i + 1] - cand_off[i] > s->d.max_cand) return GRIM_E_ARG;
    }
    const uint64_t nc = cand_off[n_reads];
    if (!chunk && nc > s->d.max_cand) return GRIM_E_ARG;
    if (nc && !cand) return GRIM_E_ARG;
    for (uint64_t k = 0; k < nc; ++k)
      if (cand[k] < 0 || (uint64_t)cand[k] >= s->ix.num_bins) return GRIM_E_BAD_CANDIDATE;
  } else if (cand || cand_off) {
    return GRIM_E_ARG;
  }
  // pieces: consecutive reads; a piece's bytes are [smallest offset, largest end)
  pieces->clear();
  Piece p;
  uint64_t lo = 0, hi = 0;
  auto close_piece = [&](uint32_t end) {
    p.n_reads = end - p.read0;
    p.byte0 = p.n_reads ? lo : 0;
    p.n_bases = p.n_reads ? hi - lo : 0;
    p.cand0 = s->cand_mode ? cand_off[p.read0] : 0;
    p.n_cand = s->cand_mode ? cand_off[end] - p.cand0 : 0;
    pieces->push_back(p);
  };
  p.read0 = 0;
  for (uint32_t i = 0; i < n_reads; ++i) {
    const uint64_t o = offsets[i], end = o + lens[i];
    if (i > p.read0) {
      const uint64_t nlo = std::min(lo, o), nhi = std::max(hi, end);
      const bool full = chunk && (i - p.read0 >= chunk || nhi - nlo > s->d.max_bases ||
                                  (s->cand_mode && cand_off[i + 1] - cand_off[p.read0] >
                                                       s->d.max_cand));
      if (full) {
        close_piece(i);
        p = Piece{};
        p.read0 = i;
        lo = o;
        hi = end;
        continue;
      }
      lo = nlo;
      hi = nhi;
    } else {
      lo = o;
      hi = end;
    }
  }
  close_piece(n_reads);
  return GRIM_OK;
}

}  // namespace

extern "C" {

int grim_server_create(const grim_index* idx, const grim_server_desc* desc, grim_server** out) {
  if (!out) return GRIM_E_ARG;
  *out = nullptr;
  if (!idx || !desc || desc->slots == 0 || desc->max_reads == 0 || desc->max_bases == 0 ||
      desc->cap == 0)
    return GRIM_E_ARG;
  if (desc->flags & ~GRIM_PLAN_CANDIDATES) return GRIM_E_ARG;
  const bool cand_mode = (desc->flags & GRIM_PLAN_CANDIDATES) != 0;
  if (cand_mode && desc->max_cand == 0) return GRIM_E_ARG;
  if (desc->max_chunk_reads > desc->max_reads) return GRIM_E_ARG;
  grim_server* s = new (std::nothrow) grim_server{};
  if (!s) return GRIM_E_NOMEM;
  s->idx = idx;
  s->d = *desc;
  s->cand_mode = cand_mode;
  int rc = grim_index_info(idx, &s->ix);
  if (rc == GRIM_OK && cudaGetDevice(&s->device) != cudaSuccess) rc = GRIM_E_CUDA;
  grim_plan_desc pd{};
  pd.max_reads = desc->max_reads;
  pd.max_e = desc->max_e;
  pd.max_bases = desc->max_bases;
  pd.max_cand = cand_mode ? desc->max_cand : 0;
  pd.cap = desc->cap;
  pd.flags = GRIM_PLAN_HOST_IO | (cand_mode ? GRIM_PLAN_CANDIDATES : 0u);
  pd.cand_unroll = desc->cand_unroll;
  // as many slots as asked for and as the device-memory budget holds
  for (uint32_t i = 0; rc == GRIM_OK && i < desc->slots; ++i) {
    Slot sl;
    rc = grim_plan_create(idx, &pd, &sl.plan);
    if (rc != GRIM_OK) break;
    const uint64_t b = grim_plan_device_bytes(sl.plan);
    if (desc->mem_budget && s->device_bytes + b > desc->mem_budget) {
      grim_plan_free(sl.plan);
      if (s->slots.empty()) rc = GRIM_E_NOMEM;
      break;
    }
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      grim_plan_free(sl.plan);
      rc = GRIM_E_CUDA;
      break;
    }
    grim_plan_buffers_get(sl.plan, &sl.buf);
    s->device_bytes += b;
    s->slots.push_back(sl);
  }
  if (rc != GRIM_OK) {
    destroy_slots(s);
    delete s;
    return rc;
  }
  s->st.slots = (uint32_t)s->slots.size();
  s->st.device_bytes = s->device_bytes;
  try {
    s->worker = std::thread([s] { s->run(); });
  } catch (...) {
    destroy_slots(s);
    delete s;
    return GRIM_E_NOMEM;
  }
  *out = s;
  return GRIM_OK;
}

int grim_server_submit(grim_server* s, const char* reads, const uint64_t* offsets,
                       const uint32_t* lens, uint32_t n_reads, const uint16_t* e,
                       const int32_t* cand, const uint64_t* cand_off, uint64_t* ticket) {
  if (!s || !ticket) return GRIM_E_ARG;
  *ticket = 0;
  const uint64_t t0 = now_ns();
  std::unique_ptr<Request> r(new (std::nothrow) Request);
  if (!r) return GRIM_E_NOMEM;
  try {
    int rc = validate(s, reads, offsets, lens, n_reads, e, cand, cand_off, &r->pieces);
    if (rc != GRIM_OK) return rc;
    uint64_t nb = 0;
    for (uint32_t i = 0; i < n_reads; ++i) nb = std::max(nb, offsets[i] + lens[i]);
    r->n_reads = n_reads;
    r->reads.assign(reads, reads + nb);
    r->offsets.assign(offsets, offsets + n_reads);
    r->lens.assign(lens, lens + n_reads);
    r->e.assign(e, e + n_reads);
    if (s->cand_mode) {
      r->cand.assign(cand, cand + cand_off[n_reads]);
      r->cand_off.assign(cand_off, cand_off + n_reads + 1);
    }
  } catch (...) {
    return GRIM_E_NOMEM;
  }
  for (Piece& p : r->pieces) p.req = r.get();
  r->pieces_left = (uint32_t)r->pieces.size();
  r->info.n_reads = n_reads;
  r->info.t_submit_ns = t0;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->fatal != GRIM_OK) return s->fatal;
    if (s->d.max_queued_reads && s->queued_reads + n_reads > s->d.max_queued_reads &&
        !s->queue.empty())
      return GRIM_E_BUSY;
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    for (Piece& p : r->pieces) s->queue.push_back(&p);
    s->queued_reads += n_reads;
    s->st.submitted++;
    s->reqs.emplace(r->ticket, std::move(r));
  }
  s->cv_work.notify_one();
  return GRIM_OK;
}

int grim_server_wait(grim_server* s, uint64_t ticket, int64_t timeout_us) {
  if (!s) return GRIM_E_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->reqs.find(ticket) == s->reqs.end()) return GRIM_E_ARG;
  // look the ticket up on every wake-up: another thread may take it meanwhile
  auto ready = [&] {
    auto it = s->reqs.find(ticket);
    return it == s->reqs.end() || it->second->done;
  };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
    return GRIM_E_NOT_READY;
  }
  return s->reqs.find(ticket) == s->reqs.end() ? GRIM_E_ARG : GRIM_OK;
}

int grim_server_take(grim_server* s, uint64_t ticket, uint32_t* out_read, uint32_t* out_bin,
                     uint8_t* out_count, uint64_t cap, grim_request_info* info) {
  if (!s) return GRIM_E_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return GRIM_E_ARG;
  Request* r = it->second.get();
  if (!r->done) return GRIM_E_NOT_READY;
  if (info) *info = r->info;
  if (r->status != GRIM_OK) {
    const int rc = r->status;
    s->reqs.erase(it);
    return rc;
  }
  if (r->n_out > cap) return GRIM_E_OVERFLOW;  // kept: take again with room for n_out
  if (r->n_out && (!out_read || !out_bin || !out_count)) return GRIM_E_ARG;
  if (r->n_out) {
    std::memcpy(out_read, r->out_read.data(), r->n_out * sizeof(uint32_t));
    std::memcpy(out_bin, r->out_bin.data(), r->n_out * sizeof(uint32_t));
    std::memcpy(out_count, r->out_count.data(), r->n_out);
  }
  s->reqs.erase(it);
  return GRIM_OK;
}

int grim_server_cancel(grim_server* s, uint64_t ticket) {
  if (!s) return GRIM_E_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || it->second->done) return GRIM_E_ARG;
  Request* r = it->second.get();
  // a request some of whose pieces have reached the device completes normally
  for (const Piece& p : r->pieces)
    if (p.started) return GRIM_E_NOT_READY;
  for (auto q = s->queue.begin(); q != s->queue.end();) {
    if ((*q)->req == r) {
      s->queued_reads -= (*q)->n_reads;
      q = s->queue.erase(q);
    } else {
      ++q;
    }
  }
  r->status = GRIM_E_CANCELLED;
  r->done = true;
  r->info.status = GRIM_E_CANCELLED;
  r->info.t_done_ns = now_ns();
  r->release_inputs();
  s->st.cancelled++;
  s->cv_done.notify_all();
  return GRIM_OK;
}

int grim_server_stats_get(grim_server* s, grim_server_stats* out) {
  if (!s || !out) return GRIM_E_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->st;
  out->queued_reads = s->queued_reads;
  out->queued_requests = s->queue.size();
  return GRIM_OK;
}

void grim_server_free(grim_server* s) {
  if (!s) return;
  {
    // requests not yet on the device are dropped; batches in flight finish,
    // then the scheduler returns
    std::lock_guard<std::mutex> g(s->mu);
    for (Piece* p : s->queue) {
      p->req->status = GRIM_E_CANCELLED;
      p->req->done = true;
    }
    s->queue.clear();
    s->queued_reads = 0;
    s->stop = true;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  destroy_slots(s);
  delete s;
}

}  // extern "C"
