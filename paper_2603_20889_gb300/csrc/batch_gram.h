// Grouped tensor-core Gram passes of the batched form (see batch_gram.cu).
#pragma once

#include "gram_launch.cuh"

namespace ql {

// One Gram-method problem of a grouped launch: its single-call arguments (float storage has
// the same layout), the first work index of its chunks in the launch and their number, and
// the tensor maps of its columns for the pipelined first pass (see pipe_tensor_maps).
struct GramGroupItem {
  GramArgs<double> args;
  int64_t work_begin;
  int nchunks;
  int tma;          // tmA (and tmB for least squares) are valid
  CUtensorMap tmA;  // 64-byte aligned: the item array is uploaded as it is laid out here
  CUtensorMap tmB;
};

// One persistent launch over `count` items (total work = their chunks) of column class nc
// (16, 32 or 64) and storage dtype, for pass 1 (Gram of X) or 2 (Gram of X M).
ql_status gram_group_launch(int nc, int dtype, int pass, int* counter, const GramGroupItem* items, int count,
                            int64_t total, cudaStream_t st);
// Rows per tile of the grouped kernels of column class nc.
int gram_group_tile_rows(int nc);

}  // namespace ql
