// Instantiates the Gram-pass kernels for float storage with ArithDF arithmetic.
#include "gram_launch.cuh"

namespace ql {
template ql_status gram_dispatch<float, ArithDF>(const GramCall&, const GramWs&, int);
}  // namespace ql
