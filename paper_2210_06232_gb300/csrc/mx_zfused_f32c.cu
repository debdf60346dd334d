// Fused z pass, FP32, the lengths 3 * 2^a up to 48 (explicit instantiations).
#include "mx_zfused.cuh"

namespace mx {
#define X(n) template MX_ZF_SIG(float, n, CoefHL);
X(6) X(12) X(24) X(48)
#undef X
}  // namespace mx
