// Fused z pass, FP32, the lengths 3 * 2^a from 96 (explicit instantiations).
#include "mx_zfused.cuh"

namespace mx {
#define X(n) template MX_ZF_SIG(float, n, CoefHL);
X(96) X(192) X(384)
#undef X
}  // namespace mx
