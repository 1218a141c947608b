// Optional per-stage CUDA-event timing used by the C ABI (pc_profile_*).
#pragma once
#include <cuda_runtime.h>

namespace pc {

enum Stage {
  kStInit = 0, kStStats, kStConsts, kStCompress, kStCodebook, kStBlockbits, kStChunkscan, kStPack,
  kStDecTables, kStDecScan, kStHuffDecode, kStRecon, kStTrain, kNumStages
};

// Records an event pair around a launch when profiling is on.
struct ProfScope {
  ProfScope(int stage, cudaStream_t s);
  ~ProfScope();
  int stage_, slot_;
  cudaStream_t s_;
};

// Called after a call synchronized its stream: folds the recorded pairs into the sums.
void prof_collect();
bool prof_on();

}  // namespace pc
