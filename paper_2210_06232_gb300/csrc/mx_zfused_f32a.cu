// Fused z pass, FP32, powers of two up to 64 (explicit instantiations).
#include "mx_zfused.cuh"

namespace mx {
#define X(n) template MX_ZF_SIG(float, n, CoefHL);
X(2) X(4) X(8) X(16) X(32) X(64)
#undef X
}  // namespace mx
