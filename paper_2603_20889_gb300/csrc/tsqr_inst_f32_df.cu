// Instantiates the TSQR kernels for float storage with ArithDF arithmetic.
#include "tsqr_launch.cuh"

namespace ql {
template ql_status dispatch<float, ArithDF>(const TsqrCall&, const TreeView&, int);
}  // namespace ql
