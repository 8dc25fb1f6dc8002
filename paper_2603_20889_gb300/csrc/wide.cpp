// QR of matrices wider than 64 columns: the hybrid of block Gram-Schmidt and TSQR panels
// that the paper's outlook names for n beyond the very-skinny regime.
//
// Panels of at most 64 columns, left to right.  Panel b is copied into a working block W,
// projected twice (ql_project_out) against every earlier panel's Q -- the coefficients land
// directly in R's off-diagonal blocks --, factored by TSQR (R's diagonal block) and turned
// into its Q by Q = W R_bb^{-1} (ql_q_from_r).  Everything runs on the caller's stream; no
// host synchronisation and no allocation (the caller's workspace holds W and the scratch of
// the three calls).
#include <cstdint>

#include <cuda_runtime.h>

#include "internal.h"

namespace ql {

constexpr int kWidePanel = 64;

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

constexpr int64_t kWideMaxN = 4096;

struct WideLayout {
  size_t w_off, proj_off, proj_bytes, tsqr_off, tsqr_bytes, info_off, bytes;
};

static bool wide_layout(int64_t m, int64_t n, ql_dtype dtype, WideLayout* L) {
  if (m < 0 || n < 1 || n > kWideMaxN || (dtype != QL_F64 && dtype != QL_F32)) return false;
  const size_t el = dtype == QL_F64 ? 8 : 4;
  const size_t w = align256((size_t)(m > 1 ? m : 1) * kWidePanel * el);
  const size_t pb = ql_project_workspace_bytes(kWidePanel, kWidePanel);
  const size_t tb = ql_workspace_bytes(QL_TSQR, m, kWidePanel, dtype);
  if (!pb || !tb) return false;
  L->w_off = 0;
  L->proj_off = w;
  L->proj_bytes = align256(pb);
  L->tsqr_off = L->proj_off + L->proj_bytes;
  L->tsqr_bytes = align256(tb);
  L->info_off = L->tsqr_off + L->tsqr_bytes;  // one {status, index} per TSQR and per Q call
  L->bytes = L->info_off + align256((size_t)4 * ((n + kWidePanel - 1) / kWidePanel) * sizeof(int32_t));
  return true;
}

}  // namespace ql

using namespace ql;

extern "C" {

size_t ql_qr_wide_workspace_bytes(int64_t m, int64_t n, ql_dtype dtype) {
  WideLayout L;
  return wide_layout(m, n, dtype, &L) ? L.bytes : 0;
}

ql_status ql_qr_wide(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R, int64_t ldr,
                     void* Q, int64_t ldq, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
  const int64_t lmin = m > 1 ? m : 1;
  if (m < 0 || n < 1 || (dtype != QL_F64 && dtype != QL_F32) || ldx < lmin || ldq < lmin || ldr < n || !R ||
      (m > 0 && (!X || !Q)))
    return QL_ERR_ARG;
  WideLayout L;
  if (!wide_layout(m, n, dtype, &L)) return QL_ERR_ARG;
  if (!ws || ws_bytes < L.bytes) return QL_ERR_WORKSPACE;
  const size_t el = dtype == QL_F64 ? 8 : 4;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = static_cast<unsigned char*>(ws);
  unsigned char* W = base + L.w_off;
  void* pws = base + L.proj_off;
  void* tws = base + L.tsqr_off;
  int32_t* infos = reinterpret_cast<int32_t*>(base + L.info_off);
  const unsigned char* Xb = static_cast<const unsigned char*>(X);
  unsigned char* Qb = static_cast<unsigned char*>(Q);
  // R starts as zero: its strictly lower blocks are never written by the panels
  for (int64_t j = 0; j < n; ++j)
    if (cudaMemsetAsync(R + j * ldr, 0, (size_t)n * sizeof(double), st) != cudaSuccess) return QL_ERR_CUDA;
  const int panels = (int)((n + kWidePanel - 1) / kWidePanel);
  if (cudaMemsetAsync(infos, 0, (size_t)4 * panels * sizeof(int32_t), st) != cudaSuccess) return QL_ERR_CUDA;
  for (int64_t c0 = 0; c0 < n; c0 += kWidePanel) {
    int32_t* pinfo = infos + 4 * (c0 / kWidePanel);  // [TSQR status, index, Q status, index]
    const int64_t nb = n - c0 < kWidePanel ? n - c0 : kWidePanel;
    // W <- X(:, c0 : c0 + nb)
    if (m > 0 && cudaMemcpy2DAsync(W, (size_t)lmin * el, Xb + (size_t)c0 * ldx * el, (size_t)ldx * el,
                                   (size_t)m * el, (size_t)nb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return QL_ERR_CUDA;
    // project against every earlier panel's Q; coefficients -> R(a0 : a0 + ka, c0 : c0 + nb)
    for (int64_t a0 = 0; a0 < c0; a0 += kWidePanel) {
      const int64_t ka = c0 - a0 < kWidePanel ? c0 - a0 : kWidePanel;
      ql_status s = ql_project_out(m, ka, Qb + (size_t)a0 * ldq * el, ldq, nb, W, lmin, dtype, W, lmin,
                                   R + c0 * ldr + a0, ldr, pws, L.proj_bytes, stream);
      if (s) return s;
    }
    // R(c0 : c0 + nb, c0 : c0 + nb) <- R of W (TSQR);  Q(:, c0 : c0 + nb) <- W R_bb^{-1}
    ql_status s = ql_tsqr_qless(m, nb, W, dtype, lmin, R + c0 * ldr + c0, ldr, pinfo, tws, L.tsqr_bytes, stream);
    if (s) return s;
    s = ql_q_from_r(m, nb, W, dtype, lmin, R + c0 * ldr + c0, ldr, Qb + (size_t)c0 * ldq * el, ldq, pinfo + 2,
                    stream);
    if (s) return s;
  }
  return info ? first_status_async(info, infos, 2 * panels, st) : QL_OK;
}

}  // extern "C"
