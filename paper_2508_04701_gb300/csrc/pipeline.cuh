// Internal interface of the fused pipeline, shared by the single-query and batched paths.
#pragma once

#include "tables.cuh"

namespace sirius {

enum { kAggAuto = 0, kAggSmem = 1, kAggGlobal = 2 };
constexpr int64_t kSmemAggMaxBytes = 96 * 1024;  // shared-memory aggregates up to 3072 slots

struct PipeHeader {
  int32_t status;
  uint32_t blocks_done;          // finalize blocks that have finished
  unsigned long long distinct;   // group slots claimed by the build
  unsigned long long groups;     // G
  unsigned long long pad[29];
};
static_assert(sizeof(PipeHeader) == 256, "pipeline header is 256 bytes");

// Scratch layout of one pipeline: [PipeHeader | JoinHeader + join slots | group keys | aggs].
struct PipeLayout {
  int key_width = 4;
  int64_t jcap = 0, gcap = 0;
  size_t off_phdr = 0, off_join = 0, off_gkeys = 0, off_aggs = 0, total = 0;
};

struct PipeOut {
  int64_t* keys;
  int64_t* sum;
  int64_t* count;
  int64_t* min;
  int64_t* max;
  int64_t cap;
  int64_t* d_groups;
  int32_t* d_status;
};

PipeLayout pipe_layout(const sirius_pipeline_desc* q);
sirius_status validate_desc(const sirius_pipeline_desc* q);
int choose_mode(const sirius_pipeline_desc* q, const PipeLayout& L);
sirius_status pipe_launch(const sirius_pipeline_desc* q, const PipeLayout& L, char* base,
                          const PipeOut& out, cudaStream_t s, bool build);
sirius_status pipe_sync_result(const PipeLayout& L, char* base, sirius_result* r, cudaStream_t s);

}  // namespace sirius
