// Map-reduce launch that allocates nothing: pyc_reduce_launch_static.
//
// Some callers cannot call cudaMalloc where they launch: programs that reserve
// all device memory at start-up and must not allocate afterwards (a fixed
// memory footprint), hosts whose device memory is owned by an outside memory
// manager, and latency-critical loops where an allocation would synchronise
// the device and break the time budget.  pyc_reduce_launch allocates its workspace (the
// per-CTA partials and the finishing ticket) on the first launch per stream;
// this variant instead uses the file-scope array below, which every GPU that
// loads the library holds until the process exits.
//
// The reduction itself is the same generated kernel with the same chunk plan
// as pyc_reduce_launch, so the two give identical results for the same input
// and tuning.
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "cudrv.h"
#include "handles.h"

namespace {

// Partials for the largest chunk plan (kMaxChunks slots of the widest, 16-byte
// accumulator) followed by the 4-byte ticket, padded to 256 bytes.
constexpr size_t kPartBytes = (size_t)pyc::kMaxChunks * 16;
constexpr size_t kScratchBytes = kPartBytes + 256;

// One scratch area per device.  In host code this name is only a stand-in for
// the device object; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char pyc_static_scratch[kScratchBytes];

// Scratch address per context.  The array's address is a property of the
// module instance in a context, not of the device: two contexts on one device
// (the primary one and one a caller created with cuCtxCreate) each hold their
// own copy of the library's device module, so each gets its own entry.  Like
// the library's other per-context state (modules, workspaces), entries are
// keyed by the context handle.
std::mutex g_mu;
std::map<CUcontext, void*> g_scratch;

// Device address of the scratch area in `ctx`, which must be current; the first
// call in a context looks it up (this loads the library's own device module
// there).
void* scratch_address(CUcontext ctx) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_scratch.find(ctx);
  if (it != g_scratch.end()) return it->second;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, pyc_static_scratch);
  if (e != cudaSuccess || !p)
    pyc::fail(PYC_E_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                              cudaGetErrorString(e));
  g_scratch.emplace(ctx, p);
  return p;
}

int variant_index(const pyc::Variant& v) {
  const auto& all = pyc::all_variants();
  for (size_t k = 0; k < all.size(); ++k)
    if (all[k].vec_bytes == v.vec_bytes && all[k].unroll == v.unroll) return (int)k;
  return -1;
}

// Per-context set-up of the handle: kernel handles and occupancy of every
// (variant, block) pair, so later calls only look values up.
void setup_handle(pyc_reduce* h, CUcontext ctx) {
  if (h->static_ctx == ctx) return;
  const auto& all = pyc::all_variants();
  const int sms = pyc::current_device_props().sm_count;
  for (size_t k = 0; k < all.size(); ++k) {
    CUfunction f = h->mod->function(h->kname("pyc_reduce", all[k]));
    h->static_fn[k] = f;
    for (int b = 1; b <= 16; ++b) {
      int nb = 0;
      PYC_CU(pyc::drv().cuOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 32 * b, 0));
      h->static_resident[k][b] = nb * sms;  // 0: this block size cannot be resident
    }
  }
  h->static_ctx = ctx;
}

}  // namespace

using namespace pyc;

PYC_API pyc_status pyc_reduce_launch_static(pyc_reduce_t h, int64_t n, void* const* ptrs,
                                            const void* scalars, void* d_out,
                                            pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    if (n < 0) fail(PYC_E_ARG, "n must be >= 0");
    if (!d_out) fail(PYC_E_ARG, "d_out is NULL");
    if (reinterpret_cast<uintptr_t>(d_out) % (uintptr_t)(h->gen.out_bytes < 8 ? h->gen.out_bytes : 8))
      fail(PYC_E_ARG, "d_out is not aligned to the result type");
    if (h->gen.acc_bytes > 16) fail(PYC_E_INTERNAL, "accumulator wider than the static slots");
    CUcontext ctx = ensure_context();
    char* scratch = static_cast<char*>(scratch_address(ctx));

    std::lock_guard<std::mutex> lk(h->static_mu);
    setup_handle(h, ctx);
    LaunchCfg cfg = choose_cfg(*h, n, true);
    int vi = variant_index(cfg.v);
    if (vi < 0 || cfg.block < 32 || cfg.block > 512 || cfg.block % 32)
      fail(PYC_E_ARG, "invalid launch configuration");

    // argument struct on the stack (no host allocation either)
    unsigned char args[4096];
    const ArgSpec& spec = h->spec;
    const int nbytes = spec.params.empty() ? 4 : spec.args_bytes;
    if (nbytes > (int)sizeof(args)) fail(PYC_E_ARG, "argument list too large");
    if (spec.num_ptrs > 0 && !ptrs) fail(PYC_E_ARG, "ptrs is NULL but the spec declares arrays");
    if (spec.scalar_bytes > 0 && !scalars)
      fail(PYC_E_ARG, "scalars is NULL but the spec declares scalar parameters");
    for (int j = 0; j < nbytes; ++j) args[j] = 0;
    for (const auto& p : spec.params) {
      const unsigned char* src = p.is_ptr
          ? reinterpret_cast<const unsigned char*>(&ptrs[p.ptr_slot])
          : static_cast<const unsigned char*>(scalars) + p.scalar_offset;
      const int sz = p.is_ptr ? 8 : type_info(p.dtype).bytes;
      for (int j = 0; j < sz; ++j) args[p.args_offset + j] = src[j];
    }

    int64_t head = vector_head(spec, ptrs, cfg.v.vec_bytes, h->min_bytes, n);
    int64_t tile = (int64_t)cfg.block * (cfg.v.vec_bytes / h->min_bytes) * cfg.v.unroll;
    const int resident = h->static_resident[vi][cfg.block / 32];
    if (resident < 1) fail(PYC_E_ARG, "block size cannot be resident for this kernel");
    ChunkPlan cp = plan_chunks(n, head, tile, resident);
    size_t need = (size_t)cp.nchunks * (size_t)h->gen.acc_bytes;
    if (need > kPartBytes)
      fail(PYC_E_ARG, "reduction needs " + std::to_string(need) + " bytes of partials; the static "
                      "scratch holds " + std::to_string(kPartBytes));

    CUdeviceptr part = reinterpret_cast<CUdeviceptr>(scratch);
    CUdeviceptr ticket = part + kPartBytes;
    CUstream s = reinterpret_cast<CUstream>(stream);
    // the ticket must start at zero; the array keeps whatever the last call left
    PYC_CU(drv().cuMemsetD32Async(ticket, 0u, 1, s));
    void* params[] = {args, &n, &cp.head, &cp.chunk, &cp.nchunks, &part, &ticket, &d_out};
    PYC_CU(drv().cuLaunchKernel(h->static_fn[vi], (unsigned)cp.grid, 1, 1, (unsigned)cfg.block, 1,
                                1, 0, s, params, nullptr));
  });
}

PYC_API pyc_status pyc_reduce_static_scratch(void** d_addr, int64_t* bytes) {
  return guarded([&] {
    if (!d_addr && !bytes) fail(PYC_E_ARG, "d_addr and bytes are both NULL");
    if (bytes) *bytes = (int64_t)kScratchBytes;
    if (d_addr) *d_addr = scratch_address(ensure_context());
  });
}
