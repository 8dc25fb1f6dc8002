// Instantiates the Gram-pass kernels for double storage with ArithF64 arithmetic.
#include "gram_launch.cuh"

namespace ql {
template ql_status gram_dispatch<double, ArithF64>(const GramCall&, const GramWs&, int);
}  // namespace ql
