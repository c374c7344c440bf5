// Batched-product kernels instantiated for one field (P2013).
#include "kernels_impl.cuh"

namespace tftgb {
TFT_DEFINE_FIELD_BATCH(P2013, p2013)
}  // namespace tftgb
