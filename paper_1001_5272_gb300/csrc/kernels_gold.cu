// Kernels and launchers instantiated for one field (Goldilocks): single products
// and transforms.
#include "kernels_impl.cuh"

namespace tftgb {
TFT_DEFINE_FIELD_ENTRIES(Goldilocks, gold)
}  // namespace tftgb
