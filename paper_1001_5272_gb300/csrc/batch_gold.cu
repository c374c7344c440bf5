// Batched-product kernels instantiated for one field (Goldilocks).
#include "kernels_impl.cuh"

namespace tftgb {
TFT_DEFINE_FIELD_BATCH(Goldilocks, gold)
}  // namespace tftgb
