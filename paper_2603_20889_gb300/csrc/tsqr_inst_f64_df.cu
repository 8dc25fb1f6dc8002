// Instantiates the TSQR kernels for double storage with ArithDF arithmetic.
#include "tsqr_launch.cuh"

namespace ql {
template ql_status dispatch<double, ArithDF>(const TsqrCall&, const TreeView&, int);
}  // namespace ql
