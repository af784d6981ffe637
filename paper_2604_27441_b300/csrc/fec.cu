// Reed-Solomon erasure coding of I-frame packets (Section 3.2: an I-frame is
// cut into n data packets, r parity packets are added, and any n of the n + r
// packets rebuild it; the paper uses r = n / 2).
//
// Systematic code over GF(2^8), field polynomial x^8 + x^4 + x^3 + x^2 + 1:
// parity packet i is, byte by byte, sum_j C[i][j] data[j] with the Cauchy
// matrix C[i][j] = 1 / ((n + i) + j) (+ is XOR in the field).  Any square
// submatrix of [I; C] is invertible, so decoding inverts the n x n matrix of
// the received packets' generator rows (on the host, n <= 255) and multiplies
// it into the received packets; data packets that arrived are copied.
//
// Both directions are one kernel: out[row][:] = sum_j coef[row][j] * in[j][:]
// over GF(2^8).  A CTA owns 1 KB of one output row: it builds, in shared
// memory, the 256-entry product table of each of its k coefficients (from the
// log / exp tables), then every thread folds 4 bytes of the k input rows
// through the tables: one shared-memory lookup per byte and input row.
#include <string.h>

#include <vector>

#include "common.cuh"
#include "revo_internal.h"

namespace revo {

namespace {

constexpr uint32_t kPoly = 0x11D;
constexpr int kFecThreads = 256;

struct GfTables {
  uint8_t exp[512];  // exp[i] = x^i, doubled so exp[log a + log b] needs no mod
  uint8_t log[256];  // log[0] unused
};

const GfTables& gf_tables() {
  static const GfTables t = [] {
    GfTables g{};
    uint32_t v = 1;
    for (int i = 0; i < 255; ++i) {
      g.exp[i] = static_cast<uint8_t>(v);
      g.log[v] = static_cast<uint8_t>(i);
      v <<= 1;
      if (v & 0x100) v ^= kPoly;
    }
    for (int i = 255; i < 512; ++i) g.exp[i] = g.exp[i - 255];
    return g;
  }();
  return t;
}

uint8_t gf_mul_host(uint8_t a, uint8_t b) {
  if (!a || !b) return 0;
  const GfTables& t = gf_tables();
  return t.exp[t.log[a] + t.log[b]];
}

uint8_t gf_inv_host(uint8_t a) {
  const GfTables& t = gf_tables();
  return t.exp[255 - t.log[a]];
}

struct GfArgs {
  GfTables tab;
  const uint8_t* in;  // k rows of `words` 32-bit words
  size_t in_pitch;
  uint8_t* out;
  size_t out_pitch;
  const uint8_t* coef;  // rows x k (row-major), or null: the Cauchy parity rows of an (n, rows) code
  int k, rows, n;
  uint32_t words;
  uint16_t out_row[256];  // output row index of coefficient row i
};

__global__ void __launch_bounds__(kFecThreads) gf_matmul_kernel(const __grid_constant__ GfArgs a) {
  extern __shared__ uint8_t mt[];  // [k][256] product tables of this row's coefficients
  __shared__ uint8_t sexp[512], slog[256];
  const int i = blockIdx.y;
  for (int t = threadIdx.x; t < 512; t += kFecThreads) sexp[t] = a.tab.exp[t];
  for (int t = threadIdx.x; t < 256; t += kFecThreads) slog[t] = a.tab.log[t];
  __syncthreads();
  for (int e = threadIdx.x; e < a.k * 256; e += kFecThreads) {
    const int j = e >> 8, b = e & 255;
    uint32_t c;
    if (a.coef) {
      c = a.coef[static_cast<size_t>(i) * a.k + j];
    } else {
      const uint32_t d = static_cast<uint32_t>(a.n + i) ^ static_cast<uint32_t>(j);  // never 0: n + i >= n > j
      c = sexp[255 - slog[d]];
    }
    mt[e] = (c && b) ? sexp[slog[c] + slog[b]] : 0;
  }
  __syncthreads();
  const uint32_t w = blockIdx.x * kFecThreads + threadIdx.x;
  if (w >= a.words) return;
  uint32_t acc = 0;
  for (int j = 0; j < a.k; ++j) {
    const uint32_t x = reinterpret_cast<const uint32_t*>(a.in + static_cast<size_t>(j) * a.in_pitch)[w];
    const uint8_t* t = mt + j * 256;
    acc ^= static_cast<uint32_t>(t[x & 255]) | (static_cast<uint32_t>(t[(x >> 8) & 255]) << 8) |
           (static_cast<uint32_t>(t[(x >> 16) & 255]) << 16) | (static_cast<uint32_t>(t[x >> 24]) << 24);
  }
  reinterpret_cast<uint32_t*>(a.out + static_cast<size_t>(a.out_row[i]) * a.out_pitch)[w] = acc;
}

cudaError_t launch_gf(GfArgs& g, cudaStream_t st) {
  if (g.rows <= 0 || g.words == 0) return cudaSuccess;
  const int smem = g.k * 256;
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = ensure_smem_attr(gf_matmul_kernel, 255 * 256, attr_done);
  if (e != cudaSuccess) return e;
  const dim3 grid((g.words + kFecThreads - 1) / kFecThreads, g.rows);
  gf_matmul_kernel<<<grid, kFecThreads, smem, st>>>(g);
  return cudaGetLastError();
}

bool fec_shape_ok(int n, int r, size_t packet_bytes) {
  return n >= 1 && r >= 0 && n + r <= 256 && packet_bytes > 0 && packet_bytes % 4 == 0 &&
         packet_bytes / 4 <= 0xFFFFFFFFull;
}

}  // namespace

cudaError_t fec_encode(int n, int r, size_t packet_bytes, const uint8_t* data, size_t data_pitch, uint8_t* parity,
                       size_t parity_pitch, cudaStream_t st) {
  if (!fec_shape_ok(n, r, packet_bytes) || data_pitch % 4 || parity_pitch % 4) return cudaErrorInvalidValue;
  GfArgs g{};
  g.tab = gf_tables();
  g.in = data;
  g.in_pitch = data_pitch;
  g.out = parity;
  g.out_pitch = parity_pitch;
  g.coef = nullptr;
  g.k = n;
  g.rows = r;
  g.n = n;
  g.words = static_cast<uint32_t>(packet_bytes / 4);
  for (int i = 0; i < r; ++i) g.out_row[i] = static_cast<uint16_t>(i);
  return launch_gf(g, st);
}

size_t fec_decode_scratch_bytes(int n) { return n > 0 ? static_cast<size_t>(n) * n : 0; }

cudaError_t fec_decode(int n, int r, size_t packet_bytes, const int* present, const uint8_t* received,
                       size_t received_pitch, uint8_t* data_out, size_t out_pitch, void* scratch, cudaStream_t st) {
  if (!fec_shape_ok(n, r, packet_bytes) || received_pitch % 4 || out_pitch % 4 || !present) return cudaErrorInvalidValue;
  // Generator rows of the received packets, then their inverse (Gauss-Jordan).
  std::vector<uint8_t> m(static_cast<size_t>(n) * 2 * n, 0);
  std::vector<char> seen(static_cast<size_t>(n + r), 0);
  for (int a = 0; a < n; ++a) {
    const int p = present[a];
    if (p < 0 || p >= n + r || seen[p]) return cudaErrorInvalidValue;
    seen[p] = 1;
    uint8_t* row = &m[static_cast<size_t>(a) * 2 * n];
    if (p < n) {
      row[p] = 1;
    } else {
      for (int j = 0; j < n; ++j) row[j] = gf_inv_host(static_cast<uint8_t>((n + (p - n)) ^ j));
    }
    row[n + a] = 1;
  }
  for (int col = 0; col < n; ++col) {
    int piv = -1;
    for (int rr = col; rr < n; ++rr)
      if (m[static_cast<size_t>(rr) * 2 * n + col]) {
        piv = rr;
        break;
      }
    if (piv < 0) return cudaErrorInvalidValue;  // cannot happen for a Cauchy code
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j)
        std::swap(m[static_cast<size_t>(piv) * 2 * n + j], m[static_cast<size_t>(col) * 2 * n + j]);
    uint8_t* prow = &m[static_cast<size_t>(col) * 2 * n];
    const uint8_t inv = gf_inv_host(prow[col]);
    for (int j = 0; j < 2 * n; ++j) prow[j] = gf_mul_host(inv, prow[j]);
    for (int rr = 0; rr < n; ++rr) {
      if (rr == col) continue;
      uint8_t* row = &m[static_cast<size_t>(rr) * 2 * n];
      const uint8_t f = row[col];
      if (!f) continue;
      for (int j = 0; j < 2 * n; ++j) row[j] ^= gf_mul_host(f, prow[j]);
    }
  }
  // Data packets that arrived are copied; the missing ones are rebuilt from
  // their rows of the inverse.
  std::vector<uint8_t> coef;
  GfArgs g{};
  int miss = 0;
  std::vector<int> where(n, -1);
  for (int a = 0; a < n; ++a)
    if (present[a] < n) where[present[a]] = a;
  cudaError_t e;
  for (int d = 0; d < n; ++d) {
    if (where[d] >= 0) {
      if ((e = cudaMemcpyAsync(data_out + static_cast<size_t>(d) * out_pitch,
                               received + static_cast<size_t>(where[d]) * received_pitch, packet_bytes,
                               cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    } else {
      coef.insert(coef.end(), &m[static_cast<size_t>(d) * 2 * n + n], &m[static_cast<size_t>(d) * 2 * n + 2 * n]);
      g.out_row[miss++] = static_cast<uint16_t>(d);
    }
  }
  if (miss == 0) return cudaSuccess;
  if (!scratch) return cudaErrorInvalidValue;
  // Pageable source: the call returns once the bytes are staged.
  if ((e = cudaMemcpyAsync(scratch, coef.data(), coef.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  g.tab = gf_tables();
  g.in = received;
  g.in_pitch = received_pitch;
  g.out = data_out;
  g.out_pitch = out_pitch;
  g.coef = static_cast<const uint8_t*>(scratch);
  g.k = n;
  g.rows = miss;
  g.n = n;
  g.words = static_cast<uint32_t>(packet_bytes / 4);
  return launch_gf(g, st);
}

}  // namespace revo
