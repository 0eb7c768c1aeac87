// grim_plan: the filter as one CUDA graph over ragged batches.
//
// grim_filter decides several things on the host between launches (the
// counter depth from the batch's largest edit budget, coarse-then-exact or
// one exact pass, whether the survivors fit, the sizes of the sorts), so it
// synchronises twice per call and cannot be captured.  A plan fixes every
// launch shape up front from declared maxima (reads, read bytes, candidates,
// output capacity, edit budget) and moves the per-batch decisions onto the
// device: the batch's counts are copied into the control block at the start
// of each run, the path is chosen there by a one-thread control kernel, the
// kernels of the path not taken return at once, and the sorts and the split
// read their record counts from device memory.  The whole sequence -- one
// persistent launch per filter pass -- is captured once into a graph and
// replayed per batch with a single cudaGraphLaunch; the control block is
// copied back to pinned host memory as the graph's last node.
#include <mutex>
#include <new>

#include "grim_internal.cuh"

namespace grim {
namespace {

// the 24 bytes of Ctl::live_reads..live_bases written by each launch
struct BatchHeader {
  uint32_t n_reads;
  uint32_t path;  // written 0: the control kernel decides
  unsigned long long n_cand;
  unsigned long long n_bases;
};
static_assert(sizeof(BatchHeader) == 24, "header mirrors Ctl::live_reads..live_bases");
static_assert(offsetof(Ctl, live_cand) - offsetof(Ctl, live_reads) == 8, "header layout");
static_assert(offsetof(Ctl, live_bases) - offsetof(Ctl, live_reads) == 16, "header layout");

// Host-memory plans: the batch's inputs are read from mapped pinned host
// memory into the device buffers by the graph itself, as many bytes as the
// batch's counts say.  Segment sizes are rounded up to 16 bytes inside
// 256-byte-aligned slots on both sides.
enum : uint32_t { kCountBases = 0, kCountReads = 1, kCountCand = 2, kCountReads1 = 3 };
struct CopySeg {
  const uint4* src;
  uint4* dst;
  uint32_t unit;      // bytes per counted element
  uint32_t count_of;  // kCount*
  uint64_t cap;       // bytes the slot holds
};
constexpr int kCopySegs = 6;
struct CopyIn {
  CopySeg s[kCopySegs];
};

__global__ void k_copy_in(CopyIn a, const Ctl* c) {
  const CopySeg& g = a.s[blockIdx.y];
  if (!g.src) return;
  const uint64_t n = g.count_of == kCountBases  ? c->live_bases
                     : g.count_of == kCountCand ? c->live_cand
                     : g.count_of == kCountReads ? (uint64_t)c->live_reads
                                                 : (uint64_t)c->live_reads + 1;
  uint64_t bytes = n * g.unit;
  if (bytes > g.cap) bytes = g.cap;
  const uint64_t n16 = (bytes + 15) / 16;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16;
       i += (uint64_t)gridDim.x * blockDim.x)
    g.dst[i] = g.src[i];
}

enum : uint32_t { kCtlDecide = 1, kCtlAfterCoarse = 2, kCtlFinal = 3 };

// One thread: the per-batch decisions that grim_filter takes on the host.
__global__ void k_plan_control(Ctl* c, uint32_t op, uint32_t capable, uint32_t has_exact,
                               unsigned long long rcap, uint32_t forced) {
  if (op == kCtlDecide) {
    const uint32_t min_slack = 255u - c->max_tight;
    c->path = (capable && (forced || min_slack >= 24 || !has_exact)) ? kPathCoarse : kPathExact;
  } else if (op == kCtlAfterCoarse) {
    if (c->path == kPathCoarse) {
      c->n_surv = c->n_rec;
      if (c->n_rec > rcap) {  // too many survivors to hold
        if (has_exact) c->path = kPathExact;
        else c->status |= kStatusSurv;
      }
    }
    c->n_rec = 0;  // restart the record and work counters for the next pass
    c->item = 0;
  } else {
    c->n_final = c->n_rec;
  }
}

}  // namespace
}  // namespace grim

using namespace grim;

struct grim_plan {
  const grim_index* idx;
  grim_plan_desc d;
  bool cand_mode;
  uint32_t f;            // coarse factor (0: no coarse path)
  Layout L;
  char* dev;             // one allocation: inputs, outputs, workspace
  grim_plan_buffers buf;   // what the caller fills and reads
  grim_plan_buffers dbuf;  // what the graph reads and writes
  bool hio;                // GRIM_PLAN_HOST_IO
  char* hin;             // mapped pinned inputs (host-memory plans)
  char* hout;            // mapped pinned outputs (host-memory plans)
  CopyIn copy;
  Ctl* ctl;
  BatchHeader* header;   // pinned
  Ctl* result;           // pinned
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaEvent_t done;
  bool launched;
};

namespace {

int capture(grim_plan* p) {
  const grim_index* idx = p->idx;
  const IndexView& v = idx->v;
  const grim_plan_desc& d = p->d;
  cudaStream_t st = p->cap_stream;
  char* ws = reinterpret_cast<char*>(p->ctl);
  const Layout& L = p->L;
  const uint64_t rcap = record_capacity(d.max_reads, d.cap, p->f);
  RecordsView ra{reinterpret_cast<unsigned long long*>(ws + L.keys_a),
                 reinterpret_cast<uint8_t*>(ws + L.cnt_a), rcap};
  RecordsView rb{reinterpret_cast<unsigned long long*>(ws + L.keys_b),
                 reinterpret_cast<uint8_t*>(ws + L.cnt_b), rcap};
  ReadsView rv{reinterpret_cast<uint16_t*>(ws + L.tok), reinterpret_cast<uint32_t*>(ws + L.meta),
               d.max_reads, token_stride(v), token_copies(v, p->cand_mode)};
  const uint32_t bin_bits = v.num_bins > 1 ? bit_length(v.num_bins - 1) : 0;
  const uint32_t read_bits = d.max_reads > 1 ? bit_length((uint64_t)d.max_reads - 1) : 0;
  const bool has_exact = (idx->layouts & GRIM_LAYOUT_TOKEN_MAJOR) != 0;
  // counters deep enough for the declared largest budget
  const uint32_t ntok_max = v.max_read_len - v.q + 1;
  uint32_t max_d = v.q * d.max_e;
  if (max_d > ntok_max) max_d = ntok_max;
  const Live live{true, 0};

  prof_suspend(true);
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    prof_suspend(false);
    return GRIM_E_CUDA;
  }
  const grim_plan_buffers& B = p->dbuf;
  cudaMemsetAsync(p->ctl, 0, sizeof(Ctl), st);
  cudaMemcpyAsync(&p->ctl->live_reads, p->header, sizeof(BatchHeader), cudaMemcpyHostToDevice, st);
  if (p->hio) k_copy_in<<<dim3(64, kCopySegs), 256, 0, st>>>(p->copy, p->ctl);
  launch_tokenise(B.reads, B.offsets, B.lens, B.e, v, rv,
                  reinterpret_cast<uint16_t*>(ws + L.tok), reinterpret_cast<uint32_t*>(ws + L.meta),
                  p->ctl, st, live, d.max_e, d.max_bases);
  if (p->cand_mode) {
    launch_check_candidates(B.cand_off, d.max_reads, d.max_cand, p->ctl, st, live);
    launch_candidates(v, rv, B.cand, B.cand_off, ra, p->ctl, st, "candidates", live,
                      d.cand_unroll, true);
    k_plan_control<<<1, 1, 0, st>>>(p->ctl, kCtlFinal, 0, 0, 0, 0);
    sort_and_emit(ra, rb, d.cap, bit_length(d.max_cand ? d.max_cand - 1 : 0), ws + L.hist, true,
                  bin_bits, B.cand, B.cand_off, d.max_reads, B.out_read,
                  B.out_bin, B.out_count, st, &p->ctl->n_final, &p->ctl->live_reads);
  } else {
    bool forced = false;
    all_bins_path(idx, &forced);
    k_plan_control<<<1, 1, 0, st>>>(p->ctl, kCtlDecide, p->f != 0, has_exact, rcap, forced);
    int32_t* icand = reinterpret_cast<int32_t*>(ws + L.cand);
    uint64_t* ioff = reinterpret_cast<uint64_t*>(ws + L.cand_off);
    const uint32_t cbits =
        idx->cv.num_bins > 1 ? bit_length(idx->cv.num_bins - 1) : 0;
    if (p->f) {
      const Live coarse{true, kPathCoarse};
      launch_exhaustive(idx->cv, rv, ra, cbits, max_d, p->ctl, st, "exhaustive_coarse", coarse,
                        idx->shape);
      k_plan_control<<<1, 1, 0, st>>>(p->ctl, kCtlAfterCoarse, 1, has_exact, rcap, 0);
      const RecordsView surv = sort_records(ra, rb, rcap, read_bits + cbits, ws + L.hist, st,
                                            &p->ctl->n_surv, p->ctl, kPathCoarse);
      expand_survivors(surv.keys, rcap, cbits, p->f, d.max_reads, icand, ioff, st, p->ctl,
                       kPathCoarse);
      launch_candidates(v, rv, icand, ioff, ra, p->ctl, st, "candidates_refine", coarse,
                        d.cand_unroll);
    }
    if (has_exact) {
      const Live exact{true, kPathExact};
      launch_exhaustive(v, rv, ra, bin_bits, max_d, p->ctl, st, "exhaustive", exact, idx->shape);
    }
    k_plan_control<<<1, 1, 0, st>>>(p->ctl, kCtlFinal, 0, 0, 0, 0);
    if (p->f) {
      sort_and_emit(ra, rb, d.cap, bit_length(rcap * p->f - 1), ws + L.hist, true, bin_bits, icand,
                    ioff, d.max_reads, B.out_read, B.out_bin, B.out_count, st,
                    &p->ctl->n_final, &p->ctl->live_reads, p->ctl, kPathCoarse);
    }
    if (has_exact) {
      sort_and_emit(ra, rb, d.cap, bin_bits + read_bits, ws + L.hist, false, bin_bits, nullptr,
                    nullptr, d.max_reads, B.out_read, B.out_bin, B.out_count, st,
                    &p->ctl->n_final, &p->ctl->live_reads, p->ctl, kPathExact);
    }
  }
  cudaMemcpyAsync(p->result, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  e = cudaStreamEndCapture(st, &p->graph);
  prof_suspend(false);
  if (e != cudaSuccess) return GRIM_E_CUDA;
  e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  return e == cudaSuccess ? GRIM_OK : GRIM_E_CUDA;
}

void destroy(grim_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->done) cudaEventDestroy(p->done);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->dev);
  if (p->hin) cudaFreeHost(p->hin);
  if (p->hout) cudaFreeHost(p->hout);
  cudaFreeHost(p->header);
  cudaFreeHost(p->result);
  delete p;
}

}  // namespace

extern "C" {

int grim_plan_create(const grim_index* idx, const grim_plan_desc* desc, grim_plan** out) {
  if (!out) return GRIM_E_ARG;
  *out = nullptr;
  if (!idx || !desc || desc->max_reads == 0 || desc->max_bases == 0) return GRIM_E_ARG;
  if (desc->cap > 0xFFFFFFFFull || desc->max_e > 0xFFFFu || desc->cand_unroll > 8)
    return GRIM_E_ARG;
  if (desc->flags & ~(GRIM_PLAN_CANDIDATES | GRIM_PLAN_HOST_IO)) return GRIM_E_ARG;
  const bool cand_mode = (desc->flags & GRIM_PLAN_CANDIDATES) != 0;
  const bool hio = (desc->flags & GRIM_PLAN_HOST_IO) != 0;
  if (cand_mode && !(idx->layouts & GRIM_LAYOUT_BIN_MAJOR)) return GRIM_E_NO_LAYOUT;
  if (!cand_mode && !(idx->layouts & GRIM_LAYOUT_TOKEN_MAJOR) && !two_level_capable(idx))
    return GRIM_E_NO_LAYOUT;
  grim_plan* p = new (std::nothrow) grim_plan{};
  if (!p) return GRIM_E_NOMEM;
  p->idx = idx;
  p->d = *desc;
  p->cand_mode = cand_mode;
  p->hio = hio;
  bool forced = false;
  p->f = (!cand_mode && all_bins_path(idx, &forced) == kPathCoarse) ? idx->factor : 0;
  p->L = layout(idx->v, desc->max_reads, desc->cap, p->f, token_copies(idx->v, cand_mode));
  const uint64_t n = desc->max_reads;
  const uint64_t mc = cand_mode ? desc->max_cand : 0;
  // one device allocation: inputs, outputs, then the workspace (256-aligned)
  const uint64_t o_reads = 0;
  const uint64_t o_off = align256(o_reads + desc->max_bases);
  const uint64_t o_lens = align256(o_off + n * 8);
  const uint64_t o_e = align256(o_lens + n * 4);
  const uint64_t o_cand = align256(o_e + n * 2);
  const uint64_t o_coff = align256(o_cand + mc * 4);
  const uint64_t o_in_end = align256(o_coff + (cand_mode ? (n + 1) * 8 : 0));
  // outputs: device buffers, or mapped host memory the final kernel writes
  const uint64_t o_or = 0;
  const uint64_t o_ob = align256(o_or + desc->cap * 4);
  const uint64_t o_oc = align256(o_ob + desc->cap * 4);
  const uint64_t out_bytes = align256(o_oc + desc->cap);
  const uint64_t o_out = o_in_end;
  const uint64_t o_ws = hio ? o_in_end : o_out + out_bytes;
  const uint64_t total = o_ws + p->L.total;
  cudaError_t e = cudaMalloc(&p->dev, total);
  if (e == cudaSuccess && hio) e = cudaHostAlloc(&p->hin, o_in_end, cudaHostAllocMapped);
  if (e == cudaSuccess && hio) e = cudaHostAlloc(&p->hout, out_bytes, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaMallocHost(&p->header, sizeof(BatchHeader));
  if (e == cudaSuccess) e = cudaMallocHost(&p->result, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    destroy(p);
    return e == cudaErrorMemoryAllocation ? GRIM_E_NOMEM : GRIM_E_CUDA;
  }
  auto inputs = [&](char* b, grim_plan_buffers& f) {
    f.reads = b + o_reads;
    f.offsets = reinterpret_cast<uint64_t*>(b + o_off);
    f.lens = reinterpret_cast<uint32_t*>(b + o_lens);
    f.e = reinterpret_cast<uint16_t*>(b + o_e);
    f.cand = cand_mode ? reinterpret_cast<int32_t*>(b + o_cand) : nullptr;
    f.cand_off = cand_mode ? reinterpret_cast<uint64_t*>(b + o_coff) : nullptr;
  };
  auto outputs = [&](char* b, grim_plan_buffers& f) {
    f.out_read = reinterpret_cast<uint32_t*>(b + o_or);
    f.out_bin = reinterpret_cast<uint32_t*>(b + o_ob);
    f.out_count = reinterpret_cast<uint8_t*>(b + o_oc);
  };
  inputs(p->dev, p->dbuf);
  if (hio) {
    void* hout_dev = nullptr;
    e = cudaHostGetDevicePointer(&hout_dev, p->hout, 0);
    if (e != cudaSuccess) {
      destroy(p);
      return GRIM_E_CUDA;
    }
    outputs(static_cast<char*>(hout_dev), p->dbuf);
    inputs(p->hin, p->buf);
    outputs(p->hout, p->buf);
    void* hin_dev = nullptr;
    e = cudaHostGetDevicePointer(&hin_dev, p->hin, 0);
    if (e != cudaSuccess) {
      destroy(p);
      return GRIM_E_CUDA;
    }
    const uint64_t in_off[kCopySegs] = {o_reads, o_off, o_lens, o_e, o_cand, o_coff};
    const uint64_t in_end[kCopySegs] = {o_off, o_lens, o_e, o_cand, o_coff, o_in_end};
    const uint32_t unit[kCopySegs] = {1, 8, 4, 2, 4, 8};
    const uint32_t cnt[kCopySegs] = {kCountBases, kCountReads, kCountReads, kCountReads,
                                     kCountCand, kCountReads1};
    for (int i = 0; i < kCopySegs; ++i) {
      const bool used = i < 4 || cand_mode;
      p->copy.s[i].src = used ? reinterpret_cast<const uint4*>(static_cast<char*>(hin_dev) + in_off[i])
                              : nullptr;
      p->copy.s[i].dst = reinterpret_cast<uint4*>(p->dev + in_off[i]);
      p->copy.s[i].unit = unit[i];
      p->copy.s[i].count_of = cnt[i];
      p->copy.s[i].cap = in_end[i] - in_off[i];
    }
  } else {
    outputs(p->dev + o_out, p->dbuf);
    p->buf = p->dbuf;
  }
  p->ctl = reinterpret_cast<Ctl*>(p->dev + o_ws);
  p->header->n_reads = 0;
  p->header->path = 0;
  p->header->n_cand = 0;
  p->header->n_bases = 0;
  const int rc = capture(p);
  if (rc != GRIM_OK) {
    destroy(p);
    return rc;
  }
  *out = p;
  return GRIM_OK;
}

int grim_plan_buffers_get(const grim_plan* p, grim_plan_buffers* out) {
  if (!p || !out) return GRIM_E_ARG;
  *out = p->buf;
  return GRIM_OK;
}

int grim_plan_launch(grim_plan* p, uint32_t n_reads, uint64_t n_cand, void* stream) {
  if (!p) return GRIM_E_ARG;
  if (n_reads > p->d.max_reads || (p->cand_mode && n_cand > p->d.max_cand)) return GRIM_E_ARG;
  // the header is read by the graph's first node: wait until the previous
  // run of this plan has consumed it
  if (p->launched && cudaEventSynchronize(p->done) != cudaSuccess) return GRIM_E_CUDA;
  uint64_t n_bases = 0;
  if (p->hio) {
    // the graph copies the reads' bytes [0, n_bases): every read must lie inside
    for (uint32_t i = 0; i < n_reads; ++i) {
      const uint64_t o = p->buf.offsets[i], l = p->buf.lens[i];
      if (o > p->d.max_bases || l > p->d.max_bases - o) return GRIM_E_ARG;
      if (o + l > n_bases) n_bases = o + l;
    }
  }
  p->header->n_reads = n_reads;
  p->header->path = 0;
  p->header->n_cand = p->cand_mode ? n_cand : 0;
  p->header->n_bases = n_bases;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGraphLaunch(p->exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(p->done, st);
  p->launched = e == cudaSuccess;
  return e == cudaSuccess ? GRIM_OK : GRIM_E_CUDA;
}

int grim_plan_query(const grim_plan* p) {
  if (!p) return GRIM_E_ARG;
  if (!p->launched) return GRIM_OK;
  const cudaError_t e = cudaEventQuery(p->done);
  if (e == cudaSuccess) return GRIM_OK;
  if (e == cudaErrorNotReady) return GRIM_E_NOT_READY;
  return GRIM_E_CUDA;
}

int grim_plan_wait(grim_plan* p, uint64_t* n_out) {
  if (!p || !n_out) return GRIM_E_ARG;
  *n_out = 0;
  if (!p->launched) return GRIM_E_ARG;
  if (cudaEventSynchronize(p->done) != cudaSuccess) return GRIM_E_CUDA;
  const Ctl& h = *p->result;
  if (h.status & kStatusSurv) {
    // every passing record lies in a surviving super-bin
    *n_out = h.n_surv * p->f;
    return GRIM_E_OVERFLOW;
  }
  const int sc = status_to_code(h.status);
  if (sc != GRIM_OK) return sc;
  *n_out = h.n_final;
  return h.n_final > p->d.cap ? GRIM_E_OVERFLOW : GRIM_OK;
}

uint64_t grim_plan_device_bytes(const grim_plan* p) {
  if (!p) return 0;
  return (uint64_t)(reinterpret_cast<char*>(p->ctl) - p->dev) + p->L.total;
}

void grim_plan_free(grim_plan* p) {
  if (!p) return;
  if (p->launched) cudaEventSynchronize(p->done);
  destroy(p);
}

}  // extern "C"
