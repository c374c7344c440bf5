// Kernels and launchers instantiated for one field (P2013): single products
// and transforms.
#include "kernels_impl.cuh"

namespace tftgb {
TFT_DEFINE_FIELD_ENTRIES(P2013, p2013)
}  // namespace tftgb
