// Kronecker mode contractions on the tcgen05 tensor cores (placeholder until
// the split-BF16 kernel lands).
#include "internal.h"

namespace cola {

void kron_tc_prepare(Ctx* c, cola_linop* op, int split_terms) { (void)c; (void)op; (void)split_terms; }

template <typename T>
void kron_tc_apply(Ctx* c, const cola_linop* op, const T* X, T* Y, int64_t R, double coeff,
                   double beta, int depth, bool tr) {
  fail(COLA_ERR_UNSUPPORTED, "MIXED precision Kronecker contraction not built yet");
}
template void kron_tc_apply<float>(Ctx*, const cola_linop*, const float*, float*, int64_t, double,
                                   double, int, bool);
template void kron_tc_apply<double>(Ctx*, const cola_linop*, const double*, double*, int64_t,
                                    double, double, int, bool);

}  // namespace cola
