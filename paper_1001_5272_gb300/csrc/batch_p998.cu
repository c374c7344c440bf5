// Batched-product kernels instantiated for one field (P998).
#include "kernels_impl.cuh"

namespace tftgb {
TFT_DEFINE_FIELD_BATCH(P998, p998)
}  // namespace tftgb
