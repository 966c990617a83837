// Source generation for map and map-reduce kernels (run-time code
// generation, Sec. 3.3: types, constants and unroll counts are written into
// the source just in time; variants are kept side by side for the tuner).
#pragma once

#include <string>
#include <vector>

#include "spec.h"

namespace pyc {

// One compiled variant: vector access width in bytes and vectors per thread
// per tile.  Block size is a launch-time choice.
struct Variant {
  int vec_bytes;
  int unroll;
};

// All variants compiled into every module.
const std::vector<Variant>& all_variants();
std::string variant_suffix(const Variant& v);

// Narrowest element size among the lifted arrays (4 if there are none).
int lifted_min_bytes(const ArgSpec& spec);

struct MapGen {
  std::string source;
  int task_bytes = 0;  // size of one batched map task record
  int task_off_n = 0;
  int task_off_head = 0;
  int task_off_chunk = 0;
};

// `tag` names the kernels (pyc_map_<tag>_v16_u4, ...) so profiles tell specs apart.
MapGen generate_map(const ArgSpec& spec, const std::string& stmt_rewritten,
                    const std::string& preamble, const std::string& tag);

enum class ReduceKind { Plain, Arg, Compensated };

// Register cap of the register-lean batched reduction kernels (16-byte
// variants, suffix _r<kLeanRegs>): with it a CTA of 512 threads still fits.
constexpr int kLeanRegs = 80;

// Threads of the one CTA that combines the records of a sharded reduction.
constexpr int kCombineBlock = 256;
// Bytes of one shard record (the accumulator before the final conversion).
constexpr int kRecordBytes = 16;

struct ReduceGen {
  std::string source;      // main module: single and batched reductions
  std::string source_ext;  // extra module: sharded reduction, record combine, lean batched
  int acc_bytes = 0;
  int out_bytes = 0;
  int task_bytes = 0;       // size of one batched task record
  int task_off_n = 0;       // offsets of the fixed task fields
  int task_off_head = 0;
  int task_off_chunk = 0;
  int task_off_out = 0;
  int task_off_nchunks = 0;
  int task_off_slot0 = 0;
};

// ordered_arg: 0, or for the built-in argmin (1) / argmax (2) rule a cheaper
// fold for the vector body, where each accumulator sees increasing indices.
// emit_kernels = false leaves out the entry points (the scan reuses the core).
ReduceGen generate_reduce(const ArgSpec& spec, pyc_dtype out_dtype, ReduceKind kind,
                          const std::string& neutral, const std::string& reduce_expr,
                          const std::string& map_rewritten, const std::string& preamble,
                          const std::string& tag, int ordered_arg = 0, bool emit_kernels = true);

// Parallel prefix scan (Sec. 3.2.6): the reduction core for pass 1 (chunk
// totals; the last CTA turns them into exclusive carries) plus pass 2 (each
// chunk scanned from its carry, the output statement run per element with
// `item` = inclusive and `prev_item` = exclusive prefix).
struct ScanGen {
  std::string source;
  int acc_bytes = 0;
  int stage_elem_bytes = 0;  // bytes per tile element staged in shared memory
};
ScanGen generate_scan(const ArgSpec& spec, pyc_dtype dtype, const std::string& neutral,
                      const std::string& scan_expr, const std::string& input_rewritten,
                      const std::string& output_rewritten, const std::string& preamble,
                      const std::string& tag);

// Device-side spelling of a dtype (pyc_bf16 for BF16, ...).
std::string device_type(pyc_dtype t);

}  // namespace pyc
