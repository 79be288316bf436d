// Launch counting / event timing scope used by every kernel launcher.
#pragma once

#include <cuda_runtime.h>

namespace ash {

enum KernelKind {
  kKFind = 0,
  kKClaim,
  kKCommit,
  kKEraseMark,
  kKEraseResolve,
  kKRebuild,
  kKListActive,
  kKIota,
  kKScatterRows,
  kKGatherRows,
  kKGatherKeys,
  kKQuantize,
  kKProbe,
  kKSetCtrl,
  kKBatch,
  kKSynthKeys,
  kKNeighbors,
  kKGatherValues,
  kKDepthKeys,
  kKCompact,
  kKIntegrate,
  kKRaycast,
  kKRayRange,
  kKPartition,
  kKUnpermute,
  kKernelKinds
};

class TraceScope {
 public:
  // `launches`: kernels launched inside the scope (counted, timed together).
  TraceScope(int kind, cudaStream_t stream, int launches = 1);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  int kind_;
  cudaStream_t stream_;
  int rec_;
};

}  // namespace ash
