// Work lists for batched launches (see handles.h).
//
// Reductions: a task of at most kSmallTask elements is reduced by one warp; such
// tasks are placed first and packed blockDim/32 to a "bundle" item.  Longer tasks
// are cut into chunks of kChunkElems elements rounded up to whole tiles (the
// first chunk also takes the unaligned head), or, for a caller that asks for a
// spread, into about that many chunks of at least a given length (a lone task of
// moderate length then occupies many CTAs instead of a few); one CTA item per
// chunk, longest tasks first.  A task with several chunks owns consecutive
// partial slots and a ticket; its last chunk to finish combines the partials in
// chunk order.  Every
// choice depends only on the task itself and the launch configuration, so a
// task's result does not depend on the other tasks of the list.
//
// Maps: every task is cut into chunks the same way; one CTA item per chunk.
#include <algorithm>
#include <cstring>

#include "handles.h"

namespace pyc {

namespace {
// Chunk length of a task of len elements: kChunkElems rounded up to whole
// tiles, or with spread > 0 short enough to cut the task into about `spread`
// chunks, but never below min_chunk elements (both rounded up to whole tiles).
// A function of the task's length and the launch configuration only.
int64_t chunk_elems(const HandleBase& h, const LaunchCfg& cfg, int64_t len, int64_t spread,
                    int64_t min_chunk) {
  const int64_t tile = (int64_t)cfg.block * (cfg.v.vec_bytes / h.min_bytes) * cfg.v.unroll;
  auto whole = [&](int64_t e) { return std::max<int64_t>(tile, (e + tile - 1) / tile * tile); };
  const int64_t cap = whole(kChunkElems);
  if (spread <= 0) return cap;
  const int64_t want = std::max<int64_t>((len + spread - 1) / spread, min_chunk);
  return std::min(cap, whole(want));
}
}  // namespace

int64_t write_reduce_work(const pyc_reduce* h, const LaunchCfg& cfg,
                          const std::vector<ReduceTaskIn>& in, std::vector<unsigned char>& tasks,
                          std::vector<ReduceItem>& items, int64_t spread, int64_t min_chunk) {
  const ArgSpec& spec = h->spec;
  const ReduceGen& g = h->gen;
  const int64_t ntask = (int64_t)in.size();
  const int wpb = cfg.block / 32;
  std::vector<int64_t> small, large;
  for (int64_t t = 0; t < ntask; ++t) (in[t].n <= kSmallTask ? small : large).push_back(t);
  std::stable_sort(large.begin(), large.end(),
                   [&](int64_t a, int64_t b) { return in[a].n > in[b].n; });
  std::vector<int64_t> order(small);
  order.insert(order.end(), large.begin(), large.end());

  tasks.assign((size_t)ntask * g.task_bytes, 0);
  items.clear();
  int64_t slots = 0;
  for (int64_t t = 0; t < ntask; ++t) {
    const ReduceTaskIn& r = in[order[t]];
    const int64_t len = r.n;
    if (len < 0) fail(PYC_E_ARG, "task length must be >= 0");
    std::vector<unsigned char> args = pack_args(spec, r.ptrs, r.scalars);
    int64_t head = vector_head(spec, r.ptrs, cfg.v.vec_bytes, h->min_bytes, len);
    unsigned char* rec = &tasks[(size_t)t * g.task_bytes];
    std::memcpy(rec, args.data(), args.size());
    int64_t tchunk, nch;
    if (len <= kSmallTask) {
      tchunk = std::max<int64_t>(len, 1);
      nch = 0;
    } else {
      int64_t body = head >= 0 ? len - head : len;
      tchunk = chunk_elems(*h, cfg, len, spread, min_chunk);
      nch = (body + tchunk - 1) / tchunk;
    }
    int32_t nchunks = (int32_t)nch, slot0 = 0;
    if (nch > 1) {
      slot0 = (int32_t)slots;
      slots += nch;
    }
    std::memcpy(rec + g.task_off_n, &len, 8);
    std::memcpy(rec + g.task_off_head, &head, 8);
    std::memcpy(rec + g.task_off_chunk, &tchunk, 8);
    std::memcpy(rec + g.task_off_out, &r.out, 8);
    std::memcpy(rec + g.task_off_nchunks, &nchunks, 4);
    std::memcpy(rec + g.task_off_slot0, &slot0, 4);
  }
  if (slots > (int64_t)INT32_MAX) fail(PYC_E_ARG, "too many chunks in one batch");
  for (int64_t t = (int64_t)small.size(); t < ntask; ++t) {
    int32_t nchunks;
    std::memcpy(&nchunks, &tasks[(size_t)t * g.task_bytes + g.task_off_nchunks], 4);
    for (int32_t c = 0; c < nchunks; ++c) items.push_back({(int32_t)t, c, 1, 0});
  }
  for (int64_t t = 0; t < (int64_t)small.size(); t += wpb) {
    int32_t cnt = (int32_t)std::min<int64_t>(wpb, (int64_t)small.size() - t);
    items.push_back({(int32_t)t, -1, cnt, 0});
  }
  return slots;
}

void write_map_work(const pyc_map* h, const LaunchCfg& cfg, const std::vector<MapTaskIn>& in,
                    std::vector<unsigned char>& tasks, std::vector<MapItem>& items, int64_t spread,
                    int64_t min_chunk) {
  const ArgSpec& spec = h->spec;
  const MapGen& g = h->gen;
  tasks.assign(in.size() * (size_t)g.task_bytes, 0);
  items.clear();
  for (size_t t = 0; t < in.size(); ++t) {
    const MapTaskIn& m = in[t];
    if (m.n < 0) fail(PYC_E_ARG, "task length must be >= 0");
    std::vector<unsigned char> args = pack_args(spec, m.ptrs, m.scalars);
    int64_t head = vector_head(spec, m.ptrs, cfg.v.vec_bytes, h->min_bytes, m.n);
    unsigned char* rec = &tasks[t * g.task_bytes];
    const int64_t chunk = chunk_elems(*h, cfg, m.n, spread, min_chunk);
    std::memcpy(rec, args.data(), args.size());
    std::memcpy(rec + g.task_off_n, &m.n, 8);
    std::memcpy(rec + g.task_off_head, &head, 8);
    std::memcpy(rec + g.task_off_chunk, &chunk, 8);
    int64_t body = m.n <= 0 ? 0 : (head >= 0 ? m.n - head : m.n);
    int64_t nch = (body + chunk - 1) / chunk;
    for (int64_t c = 0; c < nch; ++c) items.push_back({(int32_t)t, (int32_t)c});
  }
}

}  // namespace pyc
