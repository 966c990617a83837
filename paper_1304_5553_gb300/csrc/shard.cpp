// Sharded map-reduce: one index range partitioned into contiguous shards, one
// per device (or per process), with a single exchange step.
//
// A map-reduce over [0, n) (Sec. 3.2.5) splits at any points: the reduce
// expression is associative and its neutral element is an identity, so each
// shard can be folded on its own device into a partial, the partials can be
// exchanged, and folding them with the same reduce expression in shard order
// gives the reduction of the whole range.  pyc_reduce_shard folds one shard
// into a 16-byte record (the accumulator before its conversion to the result
// type: a compensated sum keeps its binary64 (hi, lo) pair, an argmin its
// global index); pyc_reduce_combine folds K such records.  The exchange of
// records between processes is the caller's (e.g. an all-gather of 16 * K
// bytes); nothing here talks to another device.
#include <cstring>

#include "cudrv.h"
#include "handles.h"

namespace pyc {

namespace {

void check_record_ptr(const void* p, const char* what) {
  if (!p) fail(PYC_E_ARG, std::string(what) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % 8)
    fail(PYC_E_ARG, std::string(what) + " is not 8-byte aligned");
}

}  // namespace

void reduce_shard(pyc_reduce* h, int64_t n_total, int64_t i0, int64_t n, void* const* ptrs,
                  const void* scalars, void* d_rec, CUstream stream) {
  if (n_total < 0 || i0 < 0 || n < 0) fail(PYC_E_ARG, "n_total, i0 and n must be >= 0");
  if (i0 > n_total || n > n_total - i0) fail(PYC_E_ARG, "shard [i0, i0 + n) exceeds [0, n_total)");
  check_record_ptr(d_rec, "d_rec");
  const ArgSpec& spec = h->spec;
  // before the pointers are read for the vector head and the offsets below
  if (spec.num_ptrs > 0 && !ptrs) fail(PYC_E_ARG, "ptrs is NULL but the spec declares arrays");
  if (spec.scalar_bytes > 0 && !scalars)
    fail(PYC_E_ARG, "scalars is NULL but the spec declares scalar parameters");
  // A shard holds elements [i0, i0 + n) of every array and nothing else, so
  // the map expression may touch each array only at index i.
  for (const auto& p : spec.params)
    if (p.is_ptr && !p.lifted)
      fail(PYC_E_ARG, "array '" + p.name + "' is used other than as " + p.name +
                          "[i]; a shard holds only its own elements");
  LaunchCfg cfg = choose_cfg(*h, n, true);
  int64_t head = vector_head(spec, ptrs, cfg.v.vec_bytes, h->min_bytes, n);
  // pointers offset by -i0 elements: the kernel indexes them with global i
  std::vector<void*> adj((size_t)(spec.num_ptrs ? spec.num_ptrs : 1), nullptr);
  for (const auto& p : spec.params)
    if (p.is_ptr)
      adj[p.ptr_slot] = reinterpret_cast<void*>(reinterpret_cast<uintptr_t>(ptrs[p.ptr_slot]) -
                                                (uintptr_t)i0 * type_info(p.dtype).bytes);
  std::vector<unsigned char> args = pack_args(spec, adj.data(), scalars);
  CUfunction f = h->ext().function(h->kname("pyc_rshard", cfg.v));
  int resident = resident_ctas(f, cfg.block);
  int64_t tile = (int64_t)cfg.block * (cfg.v.vec_bytes / h->min_bytes) * cfg.v.unroll;
  ChunkPlan cp = plan_chunks(n, head, tile, resident);
  pyc_reduce::Workspace& w = reduce_workspace(h, stream);
  void* params[] = {args.data(), &n_total, &i0, &n, &cp.head, &cp.chunk, &cp.nchunks,
                    &w.part, &w.ticket, &d_rec};
  PYC_CU(drv().cuLaunchKernel(f, (unsigned)cp.grid, 1, 1, (unsigned)cfg.block, 1, 1, 0, stream,
                              params, nullptr));
}

void reduce_combine(pyc_reduce* h, int64_t k, const void* d_recs, void* d_out, CUstream stream) {
  if (k < 0) fail(PYC_E_ARG, "k must be >= 0");
  if (k > 0) check_record_ptr(d_recs, "d_recs");
  if (!d_out) fail(PYC_E_ARG, "d_out is NULL");
  if (reinterpret_cast<uintptr_t>(d_out) % (uintptr_t)std::min(h->gen.out_bytes, 8))
    fail(PYC_E_ARG, "d_out is not aligned to the result type");
  Module& m = h->ext();  // compiled (or loaded from the cache) before any GPU work
  ensure_context();
  CUfunction f = m.function("pyc_rcomb_" + h->tag);
  void* params[] = {&d_recs, &k, &d_out};
  PYC_CU(drv().cuLaunchKernel(f, 1, 1, 1, (unsigned)kCombineBlock, 1, 1, 0, stream, params,
                              nullptr));
}

}  // namespace pyc

using namespace pyc;

PYC_API pyc_status pyc_reduce_shard(pyc_reduce_t h, int64_t n_total, int64_t i0, int64_t n,
                                    void* const* ptrs, const void* scalars, void* d_rec,
                                    pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    reduce_shard(h, n_total, i0, n, ptrs, scalars, d_rec, reinterpret_cast<CUstream>(stream));
  });
}

PYC_API pyc_status pyc_reduce_combine(pyc_reduce_t h, int64_t k, const void* d_recs,
                                      void* d_out, pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    reduce_combine(h, k, d_recs, d_out, reinterpret_cast<CUstream>(stream));
  });
}
