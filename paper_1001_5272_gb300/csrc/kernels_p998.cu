// Kernels and launchers instantiated for one field (P998): single products
// and transforms.
#include "kernels_impl.cuh"

namespace tftgb {
TFT_DEFINE_FIELD_ENTRIES(P998, p998)
}  // namespace tftgb
