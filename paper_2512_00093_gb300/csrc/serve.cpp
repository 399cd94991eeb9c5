// serve.cpp -- the serving engine of libranmar (ranmar_serve_* in ranmar.h).
//
// A native continuous-batching scheduler over the library's own entry
// points.  A request asks for the next `count` outputs of stream k of
// (seed, J): the block that starts k J transitions after the LAMMPS-seeded
// state (Sec. 1), resumed at `offset`.  Every scheduler iteration takes the
// requests that arrived, in order, while the output pool and the state pool
// allow; cuts each into segments of at most `seg` outputs (one state each,
// so a long request runs on many warps); and enqueues
//   * on the engine's own stream: ONE host-to-device copy of a packed
//     staging buffer (descriptors, checksum items, jump exponents and
//     indices, new seeds, the iteration's zeroed checksum slots), the
//     seeding of new seeds, and the jumps of the segment start states
//     (Sec. 3.1 / 3.2) -- from the seed's seeded state by k J + offset +
//     j seg, or, when the stream's state is still resident at `offset`,
//     from that state by j seg;
//   * then, on the caller's stream: one persistent generation of all
//     segments, both output types (Algorithm 2); the device checksums of
//     the outputs (how they are consumed before their memory is recycled)
//     and their copy back to the pinned staging buffer.
// Up to max_inflight iterations are on the device while the host builds
// the next, and an iteration's jumps run while earlier ones generate; an
// iteration is retired (regions and states freed, the last state of each
// request kept resident, least recently used evicted first) once its event
// has completed.  Host-side structures are flat (first-fit free map,
// entry-indexed resident set with an open-addressing key table), so that
// one iteration costs the host ~13 us and no admission stalls on evictions.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ranmar.h"

namespace ranmar {
namespace host {
int cuda_fail(cudaError_t e);   // records the CUDA error string (ranmar.cu)
}  // namespace host
}  // namespace ranmar

struct ranmar_serve;

namespace {

using Clock = std::chrono::steady_clock;

constexpr uint64_t kRegionAlign = 32;          // output regions start on 128-byte lines
constexpr double kSlowLoopSeconds = 0.01;       // a loop turn longer than this is counted
// Waits for an arrival shorter than this spin instead of sleeping: a sleep
// can overrun by milliseconds on a loaded host, which would delay every
// request that arrives meanwhile.
constexpr double kSpinSeconds = 2e-3;
constexpr size_t kPlainRing = 1024;             // plain-mode requests in flight at most
constexpr size_t kFusedSumsMax = 4096;          // segments an iteration sums inside its generation

static_assert(sizeof(ranmar_request_t) == 88, "request layout");
static_assert(sizeof(ranmar_serve_seg_t) == 72, "trace layout");
static_assert(sizeof(ranmar_serve_config_t) == 40, "config layout");
static_assert(sizeof(ranmar_serve_stats_t) == 144, "stats layout");

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

int cuda_check(cudaError_t e) { return e == cudaSuccess ? RANMAR_OK : ranmar::host::cuda_fail(e); }

// ---------------------------------------------------------------------------
// First-fit allocator over [0, size) words; free blocks keyed by start and
// coalesced with both neighbours on release.
class FirstFit {
 public:
  explicit FirstFit(uint64_t size) : size_(size) {
    if (size) free_.emplace(0, size);
  }
  static uint64_t rounded(uint64_t n) {
    n = std::max<uint64_t>(n, 1);
    return (n + kRegionAlign - 1) / kRegionAlign * kRegionAlign;
  }
  bool fits_ever(uint64_t n) const { return n <= size_ && rounded(n) <= size_; }
  bool alloc(uint64_t n, uint64_t* start) {
    n = rounded(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const uint64_t st = it->first, rest = it->second - n;
      free_.erase(it);
      if (rest) free_.emplace(st + n, rest);
      *start = st;
      return true;
    }
    return false;
  }
  void release(uint64_t start, uint64_t n) {
    n = rounded(n);
    auto it = free_.emplace(start, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  uint64_t size_;
  std::map<uint64_t, uint64_t> free_;   // start -> length
};

// ---------------------------------------------------------------------------
// Jump exponents E < 2^160 as three 64-bit limbs.
struct U160 {
  uint64_t w[3];
};

// E = k J + offset; false when E (+ extra) reaches 2^160.
bool stream_exponent(uint64_t k, const uint64_t J[2], uint64_t offset, uint64_t extra,
                     U160* out) {
  using u128 = unsigned __int128;
  const u128 p0 = static_cast<u128>(k) * J[0];
  const u128 p1 = static_cast<u128>(k) * J[1];
  u128 acc = static_cast<u128>(static_cast<uint64_t>(p0)) + offset;
  const uint64_t w0 = static_cast<uint64_t>(acc);
  acc = (acc >> 64) + static_cast<uint64_t>(p0 >> 64) + static_cast<uint64_t>(p1);
  const uint64_t w1 = static_cast<uint64_t>(acc);
  acc = (acc >> 64) + static_cast<uint64_t>(p1 >> 64);   // < 2^65
  if (acc >> 32) return false;
  U160 e{{w0, w1, static_cast<uint64_t>(acc)}};
  // the largest exponent a request uses is below E + extra
  u128 s = static_cast<u128>(e.w[0]) + extra;
  s = (s >> 64) + e.w[1];
  s = (s >> 64) + e.w[2];
  if (s >> 32) return false;
  *out = e;
  return true;
}

void exponent_words(const U160& e, uint64_t add, uint32_t out[RANMAR_MAX_EXP_WORDS]) {
  using u128 = unsigned __int128;
  u128 s = static_cast<u128>(e.w[0]) + add;
  const uint64_t w0 = static_cast<uint64_t>(s);
  s = (s >> 64) + e.w[1];
  const uint64_t w1 = static_cast<uint64_t>(s);
  const uint64_t w2 = static_cast<uint64_t>((s >> 64) + e.w[2]);
  out[0] = static_cast<uint32_t>(w0);
  out[1] = static_cast<uint32_t>(w0 >> 32);
  out[2] = static_cast<uint32_t>(w1);
  out[3] = static_cast<uint32_t>(w1 >> 32);
  out[4] = static_cast<uint32_t>(w2);
}

// ---------------------------------------------------------------------------
struct StreamKey {
  int32_t seed;
  uint64_t k, J0, J1;
  bool operator==(const StreamKey& o) const {
    return seed == o.seed && k == o.k && J0 == o.J0 && J1 == o.J1;
  }
};

struct StreamKeyHash {
  size_t operator()(const StreamKey& s) const {
    uint64_t h = static_cast<uint64_t>(static_cast<uint32_t>(s.seed)) * 0x9E3779B97F4A7C15ull;
    h ^= s.k + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
    h ^= s.J0 + 0x85EBCA77C2B2AE63ull + (h << 6) + (h >> 2);
    h ^= s.J1 + 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    return static_cast<size_t>(h ^ (h >> 29));
  }
};

StreamKey key_of(const ranmar_request_t& r) { return {r.seed, r.k, r.J[0], r.J[1]}; }

// Resident stream states: which pool entry holds the state of which stream
// (and where in the stream it stands), with least-recently-used order.
// Everything is indexed by pool entry -- the key and end of the stream an
// entry holds, and the LRU links -- plus an open-addressing table from
// stream key to entry (linear probing, deletion by backward shift).  An
// eviction is a few array operations, so that taking thousands of entries
// for a long request costs microseconds, not the milliseconds of node-based
// containers.
class ResidentSet {
 public:
  void init(uint32_t entries) {
    key_.assign(entries, StreamKey{});
    end_.assign(entries, 0);
    prev_.assign(entries, -1);
    next_.assign(entries, -1);
    size_t cap = 16;
    while (cap < 2 * static_cast<size_t>(entries)) cap <<= 1;
    slots_.assign(cap, -1);
    mask_ = cap - 1;
  }
  size_t size() const { return count_; }
  bool empty() const { return count_ == 0; }
  uint64_t end_of(int32_t entry) const { return end_[entry]; }

  // The entry holding stream `k`, or -1.
  int32_t find(const StreamKey& k) const {
    for (size_t i = home(k);; i = (i + 1) & mask_) {
      const int32_t s = slots_[i];
      if (s < 0) return -1;
      if (key_[s] == k) return s;
    }
  }
  // Makes `entry` hold stream k (absent) at `end`, most recently used.
  void insert(const StreamKey& k, uint32_t entry, uint64_t end) {
    size_t i = home(k);
    while (slots_[i] >= 0) i = (i + 1) & mask_;
    slots_[i] = static_cast<int32_t>(entry);
    key_[entry] = k;
    end_[entry] = end;
    prev_[entry] = tail_;
    next_[entry] = -1;
    if (tail_ >= 0)
      next_[tail_] = static_cast<int32_t>(entry);
    else
      head_ = static_cast<int32_t>(entry);
    tail_ = static_cast<int32_t>(entry);
    ++count_;
  }
  // Removes resident `entry` (from the table and the LRU order).
  void erase(int32_t entry) {
    size_t i = home(key_[entry]);
    while (slots_[i] != entry) i = (i + 1) & mask_;
    for (size_t j = i;;) {   // backward shift over the rest of the probe run
      j = (j + 1) & mask_;
      const int32_t s = slots_[j];
      if (s < 0) break;
      const size_t h = home(key_[s]);
      const bool stays = i <= j ? (i < h && h <= j) : (i < h || h <= j);
      if (!stays) {
        slots_[i] = s;
        i = j;
      }
    }
    slots_[i] = -1;
    const int32_t p = prev_[entry], n = next_[entry];
    if (p >= 0) next_[p] = n; else head_ = n;
    if (n >= 0) prev_[n] = p; else tail_ = p;
    --count_;
  }
  // Removes and returns the least recently used entry (-1 when empty).
  int32_t pop_lru() {
    const int32_t e = head_;
    if (e >= 0) erase(e);
    return e;
  }

 private:
  size_t home(const StreamKey& k) const { return StreamKeyHash{}(k) & mask_; }
  std::vector<StreamKey> key_;
  std::vector<uint64_t> end_;
  std::vector<int32_t> prev_, next_;
  std::vector<int32_t> slots_;
  size_t mask_ = 0, count_ = 0;
  int32_t head_ = -1, tail_ = -1;
};

// One admitted request of an iteration.
struct Admitted {
  uint32_t req;       // index into the run's request array
  uint32_t first;     // its states: Iter::ents[first .. first + nseg)
  uint32_t nseg;
  bool resume;        // ents[first] is the stream's resident state at `offset`
  uint64_t region;    // first word of its output region
};

struct Iter {
  uint32_t number = 0;
  uint32_t stage = 0;
  size_t res_off = 0;   // its checksum slots in the stage buffers
  std::vector<Admitted> reqs;
  std::vector<uint32_t> ents;
};

// Pinned host + device staging of one iteration's small inputs.
struct Stage {
  unsigned char* h = nullptr;
  unsigned char* d = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;        // end of the iteration's device work
  cudaEvent_t ev_jumped = nullptr; // its start states are written
  bool busy = false;      // enqueued and not yet retired
};

// Per-segment bytes of the staging layout, at most: a checksum slot (one
// per request), a checksum item, a descriptor, one jump (exponent + two
// indices) and one new seed.
constexpr size_t kStageBytesPerSeg = 8 + sizeof(ranmar_sum_item_t) + sizeof(ranmar_desc_t) +
                                     RANMAR_MAX_EXP_WORDS * 4 + 8 + 4;
constexpr size_t kStagePad = 16 * 12;

size_t align16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

}  // namespace

// ---------------------------------------------------------------------------
struct ranmar_serve {
  ranmar_serve_config_t cfg{};
  bool host_only = false;
  bool failed = false;
  int device = -1;
  uint64_t out_words = 0;
  // device memory
  ranmar_state_t* pool = nullptr;      // state_entries states
  uint32_t* out = nullptr;             // output pool (words / float bit patterns)
  ranmar_state_t* base = nullptr;      // seeded states, one row per seed
  uint32_t* status = nullptr;
  ranmar_table_t* table = nullptr;
  ranmar_batch_t* batch = nullptr;
  std::vector<Stage> stages;
  // plain mode
  unsigned char* plain_h = nullptr;
  unsigned char* plain_d = nullptr;
  ranmar_state_t* plain_state = nullptr;
  std::vector<cudaEvent_t> plain_ev;
  // host scheduler state
  FirstFit alloc{0};
  std::vector<uint32_t> free_entries;
  ResidentSet resident;
  std::unordered_map<int32_t, uint32_t> seed_row;
  uint32_t iter_count = 0;
  ranmar_serve_stats_t stats{};
  // host-only trace
  std::vector<ranmar_serve_seg_t> trace;
  std::vector<uint32_t> trace_live_until;  // per iteration number
  // current run
  cudaEvent_t t0 = nullptr;
  Clock::time_point h0;
  ranmar_request_t* reqs = nullptr;
  cudaStream_t stream = nullptr;       // the caller's: generation, checksums, copies back
  cudaStream_t jstream = nullptr;      // the engine's: staging copy, seeding, jumps
};

namespace {

uint32_t nseg_of(const ranmar_serve& e, uint64_t count) {
  const uint64_t s = e.cfg.seg;
  const uint64_t n = count / s + (count % s != 0);
  return static_cast<uint32_t>(std::max<uint64_t>(1, std::min<uint64_t>(n, 0xFFFFFFFFull)));
}

bool fits_ever(const ranmar_serve& e, const ranmar_request_t& r) {
  const uint64_t s = e.cfg.seg;
  const uint64_t n = std::max<uint64_t>(1, r.count / s + (r.count % s != 0));
  return e.alloc.fits_ever(std::max<uint64_t>(1, r.count)) && n <= e.cfg.state_entries;
}

// Takes n free states, evicting least recently used resident states; false
// (nothing taken) when even all of them do not make n.
bool take_entries(ranmar_serve& e, uint32_t n, std::vector<uint32_t>& dst) {
  while (e.free_entries.size() < n && !e.resident.empty()) {
    e.free_entries.push_back(static_cast<uint32_t>(e.resident.pop_lru()));
    e.stats.evicted++;
  }
  if (e.free_entries.size() < n) return false;
  dst.insert(dst.end(), e.free_entries.end() - n, e.free_entries.end());
  e.free_entries.resize(e.free_entries.size() - n);
  return true;
}

// Admission: requests leave the queue head in arrival order while their
// segments fit the iteration and their output region and states fit the
// pools; a request that could never fit is refused where it stands.
void admit(ranmar_serve& e, std::deque<uint32_t>& waiting, Iter& it) {
  uint64_t nsegs = 0;
  while (!waiting.empty()) {
    ranmar_request_t& r = e.reqs[waiting.front()];
    if (!fits_ever(e, r)) {
      r.status = RANMAR_REQ_TOO_LARGE;
      waiting.pop_front();
      e.stats.rejected++;
      continue;
    }
    const uint32_t ns = nseg_of(e, r.count);
    if (!it.reqs.empty() && nsegs + ns > e.cfg.max_segments) break;
    const StreamKey key = key_of(r);
    const int32_t res = e.resident.find(key);
    const bool resume = res >= 0 && e.resident.end_of(res) == r.offset;
    uint64_t region = 0;
    if (!e.alloc.alloc(std::max<uint64_t>(1, r.count), &region)) break;
    const uint32_t first = static_cast<uint32_t>(it.ents.size());
    if (resume) {
      // out of the resident map first, so that eviction cannot pick it
      it.ents.push_back(static_cast<uint32_t>(res));
      e.resident.erase(res);
    }
    if (!take_entries(e, resume ? ns - 1 : ns, it.ents)) {
      e.alloc.release(region, std::max<uint64_t>(1, r.count));
      if (resume) {
        e.resident.insert(key, it.ents.back(), r.offset);
        it.ents.pop_back();
      }
      break;
    }
    if (resume) e.stats.resumed++;
    it.reqs.push_back({waiting.front(), first, ns, resume, region});
    waiting.pop_front();
    nsegs += ns;
  }
}

int ensure_stage(ranmar_serve& e, Stage& st, size_t bytes) {
  if (bytes <= st.cap) return RANMAR_OK;
  if (e.host_only) {
    delete[] st.h;
    st.h = new (std::nothrow) unsigned char[bytes];
    if (!st.h) return RANMAR_ENOMEM;
    st.cap = bytes;
    return RANMAR_OK;
  }
  if (st.busy) {
    int rc = cuda_check(cudaEventSynchronize(st.ev));
    if (rc) return rc;
  }
  if (st.h) cudaFreeHost(st.h);
  if (st.d) cudaFree(st.d);
  st.h = nullptr;
  st.d = nullptr;
  st.cap = 0;
  if (cudaHostAlloc(reinterpret_cast<void**>(&st.h), bytes, cudaHostAllocDefault) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&st.d), bytes) != cudaSuccess) {
    cudaGetLastError();
    return RANMAR_ENOMEM;
  }
  st.cap = bytes;
  return RANMAR_OK;
}

// New seeds of the iteration get rows of the seed table; the caller seeds
// them on the device.
int new_seed_rows(ranmar_serve& e, const Iter& it, std::vector<int32_t>& fresh, uint32_t* r0) {
  *r0 = static_cast<uint32_t>(e.seed_row.size());
  for (const Admitted& a : it.reqs) {
    const int32_t sd = e.reqs[a.req].seed;
    if (e.seed_row.count(sd)) continue;
    if (e.seed_row.size() >= e.cfg.max_seeds) return RANMAR_ERANGE;
    e.seed_row.emplace(sd, static_cast<uint32_t>(e.seed_row.size()));
    fresh.push_back(sd);
  }
  return RANMAR_OK;
}

int do_jump(ranmar_serve& e, const ranmar_state_t* src, size_t n_src, const uint32_t* idx,
            const uint32_t* exps, uint32_t words, const uint32_t* dst_idx, size_t n) {
  ranmar_stream_t s = reinterpret_cast<ranmar_stream_t>(e.jstream);
  if (e.table)
    return ranmar_jump_tab(e.table, src, n_src, idx, exps, words, e.pool, e.cfg.state_entries,
                           dst_idx, n, e.status, s);
  return ranmar_jump_scatter(src, n_src, idx, exps, words, e.pool, e.cfg.state_entries, dst_idx,
                             n, e.status, s);
}

// Builds the iteration's staging buffer and enqueues its device work.
int enqueue(ranmar_serve& e, Iter& it) {
  nvtxRangePushA("ranmar_serve.enqueue");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop_;
  const Clock::time_point tb = Clock::now();
  it.number = e.iter_count;
  it.stage = e.iter_count % static_cast<uint32_t>(e.stages.size());
  Stage& st = e.stages[it.stage];
  if (st.busy && !e.host_only) {   // not reached: a stage's last iteration has retired
    const int rs = cuda_check(cudaEventSynchronize(st.ev));
    if (rs) return rs;
  }
  const uint32_t nreq = static_cast<uint32_t>(it.reqs.size());
  std::vector<int32_t> fresh;
  uint32_t r0 = 0;
  int rc = new_seed_rows(e, it, fresh, &r0);
  if (rc) return rc;
  size_t ntot = it.ents.size(), nu = 0, nj = 0, npj = 0;
  for (const Admitted& a : it.reqs) {
    if (!e.reqs[a.req].f32) nu += a.nseg;
    if (a.resume)
      npj += a.nseg - 1;
    else
      nj += a.nseg;
  }
  const size_t m = fresh.size();
  // layout: checksum slots (zeroed here, summed into on the device, copied
  //         back) | items | descriptors (u24 ones, then f32 ones) | jump
  //         exps | base idx | dst idx | pool exps (two words) | pool base
  //         idx | pool dst idx | seeds
  size_t off = 0;
  auto place = [&off](size_t bytes) {
    const size_t at = off;
    off = align16(off + bytes);
    return at;
  };
  const size_t o_res = place(nreq * sizeof(uint64_t));
  const size_t o_items = place(ntot * sizeof(ranmar_sum_item_t));
  const size_t o_du = place(ntot * sizeof(ranmar_desc_t));
  const size_t o_je = place(nj * RANMAR_MAX_EXP_WORDS * 4);
  const size_t o_jb = place(nj * 4);
  const size_t o_jd = place(nj * 4);
  const size_t o_pe = place(npj * 2 * 4);
  const size_t o_pb = place(npj * 4);
  const size_t o_pd = place(npj * 4);
  const size_t o_sd = place(m * 4);
  rc = ensure_stage(e, st, off);
  if (rc) return rc;
  unsigned char* h = st.h;
  auto* items = reinterpret_cast<ranmar_sum_item_t*>(h + o_items);
  auto* du = reinterpret_cast<ranmar_desc_t*>(h + o_du);
  auto* df = du + nu;
  auto* je = reinterpret_cast<uint32_t*>(h + o_je);
  auto* jb = reinterpret_cast<uint32_t*>(h + o_jb);
  auto* jd = reinterpret_cast<uint32_t*>(h + o_jd);
  auto* pe = reinterpret_cast<uint32_t*>(h + o_pe);
  auto* pb = reinterpret_cast<uint32_t*>(h + o_pb);
  auto* pd = reinterpret_cast<uint32_t*>(h + o_pd);
  if (m) std::memcpy(h + o_sd, fresh.data(), m * 4);
  std::memset(h + o_res, 0, nreq * sizeof(uint64_t));
  it.res_off = o_res;
  const uint64_t seg = e.cfg.seg;
  size_t cu = 0, cf = 0, cj = 0, cp = 0;
  for (uint32_t q = 0; q < nreq; ++q) {
    const Admitted& a = it.reqs[q];
    ranmar_request_t& r = e.reqs[a.req];
    r.iteration = it.number;
    U160 E0{};
    if (!a.resume) stream_exponent(r.k, r.J, r.offset, 0, &E0);   // checked on arrival
    const uint32_t row = a.resume ? 0 : e.seed_row[r.seed];
    for (uint32_t j = 0; j < a.nseg; ++j) {
      const uint64_t js = static_cast<uint64_t>(j) * seg;
      const uint64_t cnt = r.count > js ? std::min<uint64_t>(seg, r.count - js) : 0;
      const uint32_t ent = it.ents[a.first + j];
      const bool last = j + 1 == a.nseg;
      ranmar_serve_seg_t tr{};
      if (!a.resume) {
        exponent_words(E0, js, je + cj * RANMAR_MAX_EXP_WORDS);
        jb[cj] = row;
        jd[cj] = ent;
        if (e.host_only) {
          tr.kind = RANMAR_SEG_FROM_SEED;
          tr.src = row;
          std::memcpy(tr.exp, je + cj * RANMAR_MAX_EXP_WORDS, sizeof(tr.exp));
        }
        ++cj;
      } else if (j > 0) {
        pe[2 * cp] = static_cast<uint32_t>(js);
        pe[2 * cp + 1] = static_cast<uint32_t>(js >> 32);
        pb[cp] = it.ents[a.first];
        pd[cp] = ent;
        if (e.host_only) {
          tr.kind = RANMAR_SEG_FROM_POOL;
          tr.src = it.ents[a.first];
          tr.exp[0] = pe[2 * cp];
          tr.exp[1] = pe[2 * cp + 1];
        }
        ++cp;
      } else if (e.host_only) {
        tr.kind = RANMAR_SEG_RESIDENT;
        tr.src = ent;
      }
      const ranmar_desc_t d{ent, last ? RANMAR_DESC_WRITE_BACK : 0u, a.region + js, cnt};
      if (r.f32)
        df[cf++] = d;
      else
        du[cu++] = d;
      items[r.f32 ? nu + cf - 1 : cu - 1] = {a.region + js, cnt, js, q, 0u};   // desc order
      if (e.host_only) {
        tr.iteration = it.number;
        tr.request = a.req;
        tr.entry = ent;
        tr.flags = d.flags;
        tr.out_offset = d.out_offset;
        tr.count = cnt;
        tr.index0 = js;
        e.trace.push_back(tr);
      }
    }
  }
  e.iter_count++;
  e.stats.iterations++;
  e.stats.segments += ntot;
  e.stats.base_jumps += nj;
  e.stats.pool_jumps += npj;
  e.stats.new_seeds += m;
  st.busy = true;
  if (e.host_only) {
    e.trace_live_until.push_back(0);
    e.stats.host_ns += static_cast<uint64_t>(seconds_since(tb) * 1e9);
    return RANMAR_OK;
  }
  // The staging copy, new seeds and jumps go on the engine's stream, the
  // rest on the caller's after them: the jumps of this iteration then run
  // while earlier iterations still generate.  They touch no state an
  // earlier iteration still uses: start states go to entries taken from the
  // free list, and the resident states they read were written by retired
  // iterations.
  cudaStream_t s = e.stream, js = e.jstream;
  ranmar_stream_t rs = reinterpret_cast<ranmar_stream_t>(s);
  unsigned char* d = st.d;
  rc = cuda_check(cudaMemcpyAsync(d, h, off, cudaMemcpyHostToDevice, js));
  if (rc) return rc;
  if (m) {
    rc = ranmar_seed_batch(reinterpret_cast<const int32_t*>(d + o_sd), m, e.base + r0, e.status,
                           reinterpret_cast<ranmar_stream_t>(js));
    if (rc) return rc;
  }
  if (nj) {
    rc = do_jump(e, e.base, e.cfg.max_seeds, reinterpret_cast<const uint32_t*>(d + o_jb),
                 reinterpret_cast<const uint32_t*>(d + o_je), RANMAR_MAX_EXP_WORDS,
                 reinterpret_cast<const uint32_t*>(d + o_jd), nj);
    if (rc) return rc;
  }
  if (npj) {
    rc = do_jump(e, e.pool, e.cfg.state_entries, reinterpret_cast<const uint32_t*>(d + o_pb),
                 reinterpret_cast<const uint32_t*>(d + o_pe), 2,
                 reinterpret_cast<const uint32_t*>(d + o_pd), npj);
    if (rc) return rc;
  }
  rc = cuda_check(cudaEventRecord(st.ev_jumped, js));
  if (!rc) rc = cuda_check(cudaStreamWaitEvent(s, st.ev_jumped, 0));
  if (rc) return rc;
  // Both output types in one persistent launch.  In an iteration of up to
  // kFusedSumsMax segments (a warp per segment) each segment's checksum is
  // summed by the warp that generated it, from the words it stored: one
  // launch fewer on the latency path.  A larger iteration, whose generation
  // interleaves several segments per warp, sums faster in the separate
  // checksum kernel.
  const auto* sum_items = reinterpret_cast<const ranmar_sum_item_t*>(d + o_items);
  auto* sums = reinterpret_cast<uint64_t*>(d + o_res);
  const bool fused = ntot <= kFusedSumsMax;
  rc = ranmar_batch_generate_mixed(e.batch, e.pool, e.cfg.state_entries,
                                   reinterpret_cast<const ranmar_desc_t*>(d + o_du), ntot, nu,
                                   e.out, e.out_words, fused ? sum_items : nullptr,
                                   fused ? sums : nullptr, nreq, e.status, rs);
  if (!rc && !fused)
    rc = ranmar_checksum(e.out, e.out_words, sum_items, ntot, sums, nreq, e.status, rs);
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(h + o_res, d + o_res, nreq * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, s));
  if (rc) return rc;
  rc = cuda_check(cudaEventRecord(st.ev, s));
  const uint64_t ns = static_cast<uint64_t>(seconds_since(tb) * 1e9);
  e.stats.host_ns += ns;
  e.stats.max_enqueue_ns = std::max(e.stats.max_enqueue_ns, ns);
  return rc;
}

// Whether an event has completed.  cudaErrorNotReady is consumed here so
// that the next launch check of the library does not read it back; any
// other error counts as completed, and the synchronize that follows
// reports it.
bool event_done(cudaEvent_t ev) {
  const cudaError_t q = cudaEventQuery(ev);
  if (q == cudaErrorNotReady) {
    cudaGetLastError();
    return false;
  }
  return true;
}

bool iteration_done(const ranmar_serve& e, const Iter& it) {
  if (e.host_only) return false;   // the host-only device is slow: done only when waited for
  return event_done(e.stages[it.stage].ev);
}

int retire(ranmar_serve& e, const Iter& it) {
  Stage& st = e.stages[it.stage];
  double done = 0.0;
  if (!e.host_only) {
    int rc = cuda_check(cudaEventSynchronize(st.ev));
    if (rc) return rc;
    float ms = 0.f;
    rc = cuda_check(cudaEventElapsedTime(&ms, e.t0, st.ev));
    if (rc) return rc;
    done = ms * 1e-3;
  } else {
    e.trace_live_until[it.number] = e.iter_count;
  }
  st.busy = false;
  const double host_done = seconds_since(e.h0);
  if (e.host_only) done = host_done;
  for (uint32_t q = 0; q < it.reqs.size(); ++q) {
    const Admitted& a = it.reqs[q];
    ranmar_request_t& r = e.reqs[a.req];
    r.done = done;
    r.host_done = host_done;
    r.checksum = e.host_only ? 0 : reinterpret_cast<const uint64_t*>(st.h + it.res_off)[q];
    r.status = RANMAR_REQ_DONE;
    e.alloc.release(a.region, std::max<uint64_t>(1, r.count));
    const uint32_t* ents = it.ents.data() + a.first;
    e.free_entries.insert(e.free_entries.end(), ents, ents + a.nseg - 1);
    const uint32_t last = ents[a.nseg - 1];
    const uint64_t end = r.offset + r.count;
    const StreamKey key = key_of(r);
    const int32_t cur = e.resident.find(key);
    if (cur < 0) {
      e.resident.insert(key, last, end);
    } else if (e.resident.end_of(cur) < end) {
      e.free_entries.push_back(static_cast<uint32_t>(cur));
      e.resident.erase(cur);
      e.resident.insert(key, last, end);
    } else {
      e.free_entries.push_back(last);
    }
    e.stats.outputs += r.count;
  }
  return RANMAR_OK;
}

// Arrival check: a request that can never be served is refused here.
void arrive(ranmar_serve& e, uint32_t i, std::deque<uint32_t>& waiting) {
  ranmar_request_t& r = e.reqs[i];
  r.status = RANMAR_REQ_PENDING;
  r.done = r.host_done = -1.0;
  r.checksum = 0;
  U160 E{};
  if (r.seed < 1 || r.seed > 900000000 ||
      !stream_exponent(r.k, r.J, r.offset, std::max<uint64_t>(r.count, 1), &E)) {
    r.status = RANMAR_REQ_BAD;
    e.stats.rejected++;
    return;
  }
  waiting.push_back(i);
}

// While the loop is idle: evicts a few least recently used resident states
// until a reserve of free states exists, so that a long request seldom has
// to evict thousands at once when it is admitted.
void trim(ranmar_serve& e, int budget) {
  const size_t reserve = std::min<size_t>(e.cfg.max_segments, e.cfg.state_entries / 8);
  while (budget-- > 0 && e.free_entries.size() < reserve && !e.resident.empty()) {
    e.free_entries.push_back(static_cast<uint32_t>(e.resident.pop_lru()));
    e.stats.evicted++;
  }
}

// Busy-waits (short waits) or sleeps until `until` seconds after h0,
// trimming the resident states meanwhile.
void wait_until(ranmar_serve& e, double until) {
  trim(e, 64);
  double left = until - seconds_since(e.h0);
  if (left <= 0) return;
  if (left > kSpinSeconds) {
    std::this_thread::sleep_for(std::chrono::duration<double>(std::min(left - kSpinSeconds, 1e-3)));
    return;
  }
  while (seconds_since(e.h0) < until) trim(e, 8);
}

int finish_run(ranmar_serve& e, int rc) {
  if (!e.host_only) {
    int rs = cuda_check(cudaStreamSynchronize(e.stream));
    if (!rs) rs = cuda_check(cudaStreamSynchronize(e.jstream));
    if (!rc) rc = rs;
    uint32_t st = 0;
    if (!rc) rc = cuda_check(cudaMemcpy(&st, e.status, 4, cudaMemcpyDeviceToHost));
    e.stats.status |= st;
    if (!rc && st) rc = RANMAR_ESTATUS;
  }
  if (rc) e.failed = true;
  e.reqs = nullptr;
  return rc;
}

int run_loop(ranmar_serve& e, size_t n, bool realtime, double max_wait) {
  std::deque<uint32_t> waiting;
  std::deque<Iter> inflight;
  size_t i = 0;
  Clock::time_point t_prev = Clock::now();
  uint64_t max_loop_ns = 0;
  while (i < n || !waiting.empty() || !inflight.empty()) {
    const Clock::time_point t_now = Clock::now();
    const uint64_t loop_ns = static_cast<uint64_t>(
        std::chrono::duration_cast<std::chrono::nanoseconds>(t_now - t_prev).count());
    max_loop_ns = std::max(max_loop_ns, loop_ns);
    if (loop_ns > kSlowLoopSeconds * 1e9) e.stats.slow_loops++;
    t_prev = t_now;
    const double now = std::chrono::duration<double>(t_now - e.h0).count();
    if (now > max_wait) return RANMAR_ETIME;
    while (i < n && (!realtime || e.reqs[i].t <= now)) arrive(e, static_cast<uint32_t>(i++), waiting);
    bool admitted = false;
    if (inflight.size() < e.cfg.max_inflight && !waiting.empty()) {
      Iter it;
      const Clock::time_point ta = Clock::now();
      admit(e, waiting, it);
      e.stats.max_admit_ns = std::max<uint64_t>(
          e.stats.max_admit_ns, static_cast<uint64_t>(seconds_since(ta) * 1e9));
      if (!it.reqs.empty()) {
        const int rc = enqueue(e, it);
        if (rc) return rc;
        inflight.push_back(std::move(it));
        e.stats.max_inflight = std::max<uint64_t>(e.stats.max_inflight, inflight.size());
        admitted = true;
      }
    }
    bool progressed = admitted;
    while (!inflight.empty() && (iteration_done(e, inflight.front()) ||
                                 (!admitted && (!waiting.empty() || i >= n)))) {
      const Clock::time_point tr = Clock::now();
      const int rc = retire(e, inflight.front());
      if (rc) return rc;
      e.stats.max_retire_ns = std::max<uint64_t>(
          e.stats.max_retire_ns, static_cast<uint64_t>(seconds_since(tr) * 1e9));
      inflight.pop_front();
      progressed = true;
      if (!inflight.empty() && !iteration_done(e, inflight.front())) break;
    }
    if (!progressed && realtime && i < n && waiting.empty()) {
      // idle until the next arrival; with work on the device, poll its
      // oldest iteration meanwhile so that it retires as soon as it ends
      if (inflight.empty() || e.host_only) {
        wait_until(e, e.reqs[i].t);
      } else {
        while (seconds_since(e.h0) < e.reqs[i].t && !iteration_done(e, inflight.front()))
          trim(e, 8);
      }
    }
  }
  e.stats.max_loop_ns = std::max(e.stats.max_loop_ns, max_loop_ns);
  return RANMAR_OK;
}

int start_run(ranmar_serve& e, ranmar_request_t* reqs, size_t n, ranmar_stream_t stream) {
  if (e.failed) return RANMAR_EINVAL;
  if (!reqs && n) return RANMAR_EINVAL;
  if (n >= 0xFFFFFFFFull) return RANMAR_ERANGE;
  for (size_t i = 1; i < n; ++i)
    if (!(reqs[i].t >= reqs[i - 1].t)) return RANMAR_EINVAL;   // arrival order
  e.reqs = reqs;
  e.stream = reinterpret_cast<cudaStream_t>(stream);
  if (!e.host_only) {
    int rc = cuda_check(cudaStreamSynchronize(e.stream));
    if (!rc) rc = cuda_check(cudaEventRecord(e.t0, e.stream));
    if (rc) {
      e.reqs = nullptr;
      return rc;
    }
  }
  e.h0 = Clock::now();
  return RANMAR_OK;
}

void free_device(ranmar_serve* e) {
  for (Stage& st : e->stages) {
    if (e->host_only) {
      delete[] st.h;
    } else {
      if (st.h) cudaFreeHost(st.h);
      if (st.d) cudaFree(st.d);
      if (st.ev) cudaEventDestroy(st.ev);
      if (st.ev_jumped) cudaEventDestroy(st.ev_jumped);
    }
  }
  if (!e->host_only) {
    for (cudaEvent_t ev : e->plain_ev)
      if (ev) cudaEventDestroy(ev);
    if (e->t0) cudaEventDestroy(e->t0);
    if (e->jstream) cudaStreamDestroy(e->jstream);
    cudaFree(e->pool);
    cudaFree(e->out);
    cudaFree(e->base);
    cudaFree(e->status);
    cudaFree(e->plain_d);
    cudaFree(e->plain_state);
    if (e->plain_h) cudaFreeHost(e->plain_h);
    if (e->table) ranmar_table_destroy(e->table);
    if (e->batch) ranmar_batch_destroy(e->batch);
  }
}

// Plain-mode record: one request's jump exponent and indices, seed,
// checksum item and checksum (80 bytes, pinned and on the device, one per
// request in flight; the checksum is zeroed on the host, summed into on the
// device and copied back).
struct alignas(16) PlainRec {
  uint32_t exp[RANMAR_MAX_EXP_WORDS];
  uint32_t base_idx;
  uint32_t dst_idx;
  int32_t seed;
  ranmar_sum_item_t item;
  uint64_t result;
};
static_assert(sizeof(PlainRec) == 80, "plain record");

struct PlainPending {
  uint32_t req;
  uint32_t rec;
  uint64_t region;
};

int plain_retire(ranmar_serve& e, const PlainPending& p) {
  int rc = cuda_check(cudaEventSynchronize(e.plain_ev[p.rec]));
  float ms = 0.f;
  if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, e.t0, e.plain_ev[p.rec]));
  if (rc) return rc;
  ranmar_request_t& r = e.reqs[p.req];
  r.done = ms * 1e-3;
  r.host_done = seconds_since(e.h0);
  r.checksum = (reinterpret_cast<const PlainRec*>(e.plain_h) + p.rec)->result;
  r.status = RANMAR_REQ_DONE;
  e.alloc.release(p.region, std::max<uint64_t>(1, r.count));
  return RANMAR_OK;
}

int plain_loop(ranmar_serve& e, size_t n, bool realtime, double max_wait) {
  std::deque<PlainPending> pending;
  uint32_t next_rec = 0;
  cudaStream_t s = e.stream;
  ranmar_stream_t rs = reinterpret_cast<ranmar_stream_t>(s);
  for (size_t i = 0; i < n; ++i) {
    ranmar_request_t& r = e.reqs[i];
    if (realtime)
      while (seconds_since(e.h0) < r.t) wait_until(e, r.t);
    if (seconds_since(e.h0) > max_wait) return RANMAR_ETIME;
    std::deque<uint32_t> one;
    arrive(e, static_cast<uint32_t>(i), one);
    if (one.empty()) continue;
    if (!fits_ever(e, r)) {
      r.status = RANMAR_REQ_TOO_LARGE;
      e.stats.rejected++;
      continue;
    }
    if (pending.size() == kPlainRing) {
      int rc = plain_retire(e, pending.front());
      if (rc) return rc;
      pending.pop_front();
    }
    uint64_t region = 0;
    while (!e.alloc.alloc(std::max<uint64_t>(1, r.count), &region)) {
      if (pending.empty()) return RANMAR_ERANGE;   // cannot happen: fits_ever
      int rc = plain_retire(e, pending.front());
      if (rc) return rc;
      pending.pop_front();
    }
    const uint32_t ri = next_rec;
    next_rec = (next_rec + 1) % kPlainRing;
    PlainRec* h = reinterpret_cast<PlainRec*>(e.plain_h) + ri;
    PlainRec* d = reinterpret_cast<PlainRec*>(e.plain_d) + ri;
    U160 E{};
    stream_exponent(r.k, r.J, r.offset, 0, &E);
    exponent_words(E, 0, h->exp);
    h->dst_idx = 0;
    h->seed = r.seed;
    bool fresh = false;
    auto row = e.seed_row.find(r.seed);
    if (row == e.seed_row.end()) {
      if (e.seed_row.size() >= e.cfg.max_seeds) return RANMAR_ERANGE;
      row = e.seed_row.emplace(r.seed, static_cast<uint32_t>(e.seed_row.size())).first;
      fresh = true;
    }
    h->base_idx = row->second;
    h->item = {0, r.count, 0, 0u, 0u};
    h->result = 0;
    int rc = cuda_check(cudaMemcpyAsync(d, h, sizeof(PlainRec), cudaMemcpyHostToDevice, s));
    if (!rc && fresh) rc = ranmar_seed_batch(&d->seed, 1, e.base + row->second, e.status, rs);
    if (!rc)
      rc = ranmar_jump_scatter(e.base, e.cfg.max_seeds, &d->base_idx, d->exp,
                               RANMAR_MAX_EXP_WORDS, e.plain_state, 1, &d->dst_idx, 1, e.status,
                               rs);
    if (!rc)
      rc = r.f32 ? ranmar_generate_plain_f32(e.plain_state, r.count,
                                             reinterpret_cast<float*>(e.out) + region, 0, rs)
                 : ranmar_generate_plain_u24(e.plain_state, r.count, e.out + region, 0, rs);
    if (!rc)
      rc = ranmar_checksum(e.out + region, r.count ? r.count : 1, &d->item, 1, &d->result, 1,
                           e.status, rs);
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(&h->result, &d->result, sizeof(uint64_t),
                                      cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaEventRecord(e.plain_ev[ri], s));
    if (rc) return rc;
    pending.push_back({static_cast<uint32_t>(i), ri, region});
    while (!pending.empty() && event_done(e.plain_ev[pending.front().rec])) {
      rc = plain_retire(e, pending.front());
      if (rc) return rc;
      pending.pop_front();
    }
  }
  while (!pending.empty()) {
    int rc = plain_retire(e, pending.front());
    if (rc) return rc;
    pending.pop_front();
  }
  return RANMAR_OK;
}

}  // namespace

extern "C" {

int ranmar_serve_create(const ranmar_serve_config_t* cfg, ranmar_serve_t** out) {
  if (!cfg || !out) return RANMAR_EINVAL;
  *out = nullptr;
  const ranmar_serve_config_t c = *cfg;
  if (c.seg == 0 || c.state_entries == 0 || c.max_seeds == 0 || c.max_segments == 0 ||
      c.max_inflight == 0 || (c.flags & ~(RANMAR_SERVE_SQUARE | RANMAR_SERVE_HOST_ONLY)) ||
      c.reserved != 0)
    return RANMAR_EINVAL;
  const uint64_t state_bytes = static_cast<uint64_t>(c.state_entries) * sizeof(ranmar_state_t);
  if (c.budget_bytes <= state_bytes + 4 * kRegionAlign) return RANMAR_ERANGE;
  ranmar_serve* e = new (std::nothrow) ranmar_serve();
  if (!e) return RANMAR_ENOMEM;
  e->cfg = c;
  e->host_only = (c.flags & RANMAR_SERVE_HOST_ONLY) != 0;
  e->out_words = (c.budget_bytes - state_bytes) / 4;
  e->alloc = FirstFit(e->out_words);
  // full-size tables up front: a rehash of 2^18 resident streams in the
  // middle of a run is a stall of milliseconds
  e->resident.init(c.state_entries);
  e->seed_row.reserve(c.max_seeds);
  e->free_entries.resize(c.state_entries);
  for (uint32_t q = 0; q < c.state_entries; ++q) e->free_entries[q] = c.state_entries - 1 - q;
  e->stages.resize(c.max_inflight + 1);
  const size_t stage_bytes = static_cast<size_t>(c.max_segments) * kStageBytesPerSeg + kStagePad;
  int rc = RANMAR_OK;
  if (!e->host_only) {
    rc = cuda_check(cudaGetDevice(&e->device));
    auto dalloc = [&rc](void** p, size_t bytes) {
      if (!rc && cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        rc = RANMAR_ENOMEM;
      }
    };
    dalloc(reinterpret_cast<void**>(&e->pool), state_bytes);
    dalloc(reinterpret_cast<void**>(&e->out), e->out_words * 4);
    dalloc(reinterpret_cast<void**>(&e->base),
           static_cast<size_t>(c.max_seeds) * sizeof(ranmar_state_t));
    dalloc(reinterpret_cast<void**>(&e->status), 4);
    dalloc(reinterpret_cast<void**>(&e->plain_d), kPlainRing * sizeof(PlainRec));
    dalloc(reinterpret_cast<void**>(&e->plain_state), sizeof(ranmar_state_t));
    if (!rc && cudaHostAlloc(reinterpret_cast<void**>(&e->plain_h), kPlainRing * sizeof(PlainRec),
                             cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      rc = RANMAR_ENOMEM;
    }
    if (!rc) rc = cuda_check(cudaMemset(e->status, 0, 4));
    if (!rc) rc = cuda_check(cudaEventCreate(&e->t0));
    if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&e->jstream, cudaStreamNonBlocking));
    for (Stage& st : e->stages) {
      if (!rc) rc = cuda_check(cudaEventCreate(&st.ev));
      if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&st.ev_jumped, cudaEventDisableTiming));
      if (!rc) rc = ensure_stage(*e, st, stage_bytes);
    }
    e->plain_ev.assign(kPlainRing, nullptr);
    for (cudaEvent_t& ev : e->plain_ev)
      if (!rc) rc = cuda_check(cudaEventCreate(&ev));
    if (!rc && !(c.flags & RANMAR_SERVE_SQUARE)) rc = ranmar_table_create(&e->table);
    if (!rc) rc = ranmar_batch_create(std::max<size_t>(c.max_segments, 1024), &e->batch);
  } else {
    for (Stage& st : e->stages)
      if (!rc) rc = ensure_stage(*e, st, stage_bytes);
  }
  if (rc) {
    free_device(e);
    delete e;
    return rc;
  }
  *out = e;
  return RANMAR_OK;
}

int ranmar_serve_destroy(ranmar_serve_t* e) {
  if (!e) return RANMAR_OK;
  if (!e->host_only) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != e->device) return RANMAR_EINVAL;
    cudaDeviceSynchronize();
  }
  free_device(e);
  delete e;
  return RANMAR_OK;
}

int ranmar_serve_preload(ranmar_serve_t* e, const int32_t* h_seeds, size_t n,
                         ranmar_stream_t stream) {
  if (!e || (!h_seeds && n)) return RANMAR_EINVAL;
  if (e->failed) return RANMAR_EINVAL;
  std::vector<int32_t> fresh;
  for (size_t i = 0; i < n; ++i) {
    const int32_t sd = h_seeds[i];
    if (sd < 1 || sd > 900000000) return RANMAR_EINVAL;
    if (e->seed_row.count(sd)) continue;
    if (e->seed_row.size() >= e->cfg.max_seeds) return RANMAR_ERANGE;
    fresh.push_back(sd);
    e->seed_row.emplace(sd, static_cast<uint32_t>(e->seed_row.size()));
  }
  if (fresh.empty() || e->host_only) return RANMAR_OK;
  const uint32_t r0 = static_cast<uint32_t>(e->seed_row.size() - fresh.size());
  int32_t* d = nullptr;
  int rc = RANMAR_OK;
  if (cudaMalloc(reinterpret_cast<void**>(&d), fresh.size() * 4) != cudaSuccess) {
    cudaGetLastError();
    rc = RANMAR_ENOMEM;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!rc) rc = cuda_check(cudaMemcpyAsync(d, fresh.data(), fresh.size() * 4,
                                           cudaMemcpyHostToDevice, s));
  if (!rc) rc = ranmar_seed_batch(d, fresh.size(), e->base + r0, e->status, stream);
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  cudaFree(d);
  if (rc) e->failed = true;
  return rc;
}

int ranmar_serve_run(ranmar_serve_t* e, ranmar_request_t* h_reqs, size_t n, int realtime,
                     double max_wait_s, ranmar_stream_t stream) {
  if (!e) return RANMAR_EINVAL;
  int rc = start_run(*e, h_reqs, n, stream);
  if (rc) return rc;
  nvtxRangePushA("ranmar_serve_run");
  rc = run_loop(*e, n, realtime != 0, max_wait_s);
  nvtxRangePop();
  return finish_run(*e, rc);
}

int ranmar_serve_run_plain(ranmar_serve_t* e, ranmar_request_t* h_reqs, size_t n, int realtime,
                           double max_wait_s, ranmar_stream_t stream) {
  if (!e) return RANMAR_EINVAL;
  if (e->host_only) return RANMAR_EINVAL;
  int rc = start_run(*e, h_reqs, n, stream);
  if (rc) return rc;
  nvtxRangePushA("ranmar_serve_run_plain");
  rc = plain_loop(*e, n, realtime != 0, max_wait_s);
  nvtxRangePop();
  return finish_run(*e, rc);
}

int ranmar_serve_get_stats(const ranmar_serve_t* e, ranmar_serve_stats_t* out) {
  if (!e || !out) return RANMAR_EINVAL;
  *out = e->stats;
  out->resident = e->resident.size();
  return RANMAR_OK;
}

int ranmar_serve_trace(const ranmar_serve_t* e, ranmar_serve_seg_t* h_out, size_t cap,
                       size_t* n_out) {
  if (!e || !n_out || (!h_out && cap)) return RANMAR_EINVAL;
  if (!e->host_only) return RANMAR_EINVAL;
  const size_t n = std::min(cap, e->trace.size());
  for (size_t q = 0; q < n; ++q) {
    h_out[q] = e->trace[q];
    h_out[q].live_until = e->trace_live_until[e->trace[q].iteration];
  }
  *n_out = e->trace.size();
  return RANMAR_OK;
}

}  // extern "C"
