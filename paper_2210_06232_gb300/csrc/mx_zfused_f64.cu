// Fused z pass, FP64, every length (explicit instantiations).
#include "mx_zfused.cuh"

namespace mx {
#define X(n) template MX_ZF_SIG(double, n, Coef<double>);
MX_ZF_LENS(X)
#undef X
}  // namespace mx
