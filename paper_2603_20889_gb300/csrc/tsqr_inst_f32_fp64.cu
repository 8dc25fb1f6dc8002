// Instantiates the TSQR kernels for float storage with ArithF64 arithmetic.
#include "tsqr_launch.cuh"

namespace ql {
template ql_status dispatch<float, ArithF64>(const TsqrCall&, const TreeView&, int);
}  // namespace ql
