// Fused z pass, FP32, powers of two from 128 (explicit instantiations).
#include "mx_zfused.cuh"

namespace mx {
#define X(n) template MX_ZF_SIG(float, n, CoefHL);
X(128) X(256) X(512)
#undef X
}  // namespace mx
