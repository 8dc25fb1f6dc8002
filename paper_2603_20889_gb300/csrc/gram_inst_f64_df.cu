// Instantiates the Gram-pass kernels for double storage with ArithDF arithmetic.
#include "gram_launch.cuh"

namespace ql {
template ql_status gram_dispatch<double, ArithDF>(const GramCall&, const GramWs&, int);
}  // namespace ql
