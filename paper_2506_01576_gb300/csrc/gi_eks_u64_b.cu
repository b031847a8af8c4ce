// k-ary lookup instantiations: uint64_t keys, fan-outs 16, 17, 32, 33.
#define GI_EKS_KEY uint64_t
#define GI_EKS_FN eks_point_u64_b
#define GI_EKS_LIST(X) \
  X(16, 1) \
  X(16, 16) \
  X(17, 1) \
  X(17, 4) \
  X(17, 8) \
  X(17, 16) \
  X(32, 32) \
  X(33, 8) \
  X(33, 16) \
  X(33, 32)

#include "gi_eks_inst.cuh"
