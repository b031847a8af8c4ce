// k-ary lookup instantiations: uint32_t keys, fan-outs 3, 4, 5, 8, 9.
#define GI_EKS_KEY uint32_t
#define GI_EKS_FN eks_point_u32_a
#define GI_EKS_LIST(X) \
  X(3, 1) \
  X(3, 2) \
  X(4, 1) \
  X(4, 4) \
  X(5, 1) \
  X(5, 2) \
  X(5, 4) \
  X(8, 1) \
  X(8, 8) \
  X(9, 1) \
  X(9, 2) \
  X(9, 4) \
  X(9, 8)

#include "gi_eks_inst.cuh"
