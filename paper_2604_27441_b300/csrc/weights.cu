// Host-side sources of the models' float32 master weights, for a context
// created without weight arrays: a flat little-endian file, or the documented
// random initialisation (no trained weights are published with the paper).
//
// The random initialisation draws every parameter, in the file order of
// revo.h, from one stream of uniform doubles:
//   [out][in] matrices: U(-b, b) with b = sqrt(6 / (in + out)) (Xavier-uniform),
//                       the pixel head further times 0.1;
//   LayerNorm gains:    1 + U(-0.1, 0.1);   every other vector: U(-0.02, 0.02);
// each value computed in double and rounded to float32.  The uniform doubles
// are u = (x >> 11) * 2^-53 for the 64-bit outputs x of the PCG64 generator
// (O'Neill, "PCG: A Family of Simple Fast Space-Efficient Statistically Good
// Algorithms for Random Number Generation", 2014: a 128-bit LCG with
// multiplier 0x2360ED051FC65DA44385DF649FCCF645 and the XSL-RR output), whose
// state and increment are derived from the 64-bit seed by the SeedSequence
// entropy-mixing scheme of NumPy's random module (NEP 19); U(a, b) = a + (b - a) u.
// The same definitions give the seeded weights the tests and the benchmark
// draw in Python, so a context can be created from a seed alone.
#include <math.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "model.h"

namespace revo {

namespace {

// ---- SeedSequence: hash the seed's 32-bit words into a 4-word pool, then
// expand the pool into as many state words as requested.
constexpr uint32_t kInitA = 0x43b0d7e5u, kMultA = 0x931e8875u;
constexpr uint32_t kInitB = 0x8b51f9ddu, kMultB = 0x58f38dedu;
constexpr uint32_t kMixL = 0xca01f9ddu, kMixR = 0x4973f715u;
constexpr int kPool = 4;

uint32_t hashmix(uint32_t v, uint32_t& h) {
  v ^= h;
  h *= kMultA;
  v *= h;
  return v ^ (v >> 16);
}

uint32_t mix(uint32_t x, uint32_t y) {
  uint32_t r = kMixL * x - kMixR * y;
  return r ^ (r >> 16);
}

void seed_pool(uint64_t seed, uint32_t (&pool)[kPool]) {
  std::vector<uint32_t> ent;
  // The seed as little-endian 32-bit words, without leading zero words (0 -> one word).
  do {
    ent.push_back(static_cast<uint32_t>(seed & 0xffffffffu));
    seed >>= 32;
  } while (seed);
  uint32_t h = kInitA;
  for (int i = 0; i < kPool; ++i) pool[i] = hashmix(i < static_cast<int>(ent.size()) ? ent[i] : 0u, h);
  for (int s = 0; s < kPool; ++s)
    for (int d = 0; d < kPool; ++d)
      if (s != d) pool[d] = mix(pool[d], hashmix(pool[s], h));
  for (size_t s = kPool; s < ent.size(); ++s)
    for (int d = 0; d < kPool; ++d) pool[d] = mix(pool[d], hashmix(ent[s], h));
}

void pool_state(const uint32_t (&pool)[kPool], uint32_t* out, int n) {
  uint32_t h = kInitB;
  for (int i = 0; i < n; ++i) {
    uint32_t v = pool[i % kPool];
    v ^= h;
    h *= kMultB;
    v *= h;
    out[i] = v ^ (v >> 16);
  }
}

// ---- PCG64 (128-bit state, XSL-RR output).
using u128 = unsigned __int128;

struct Pcg64 {
  u128 state = 0, inc = 0;

  static u128 mult() { return (static_cast<u128>(0x2360ED051FC65DA4ull) << 64) | 0x4385DF649FCCF645ull; }
  void step() { state = state * mult() + inc; }

  explicit Pcg64(uint64_t seed) {
    uint32_t pool[kPool], w[8];
    seed_pool(seed, pool);
    pool_state(pool, w, 8);
    // Four 64-bit words (low 32 bits first): initial state (high, low) and
    // stream selector (high, low).
    uint64_t q[4];
    for (int i = 0; i < 4; ++i) q[i] = static_cast<uint64_t>(w[2 * i]) | (static_cast<uint64_t>(w[2 * i + 1]) << 32);
    const u128 initstate = (static_cast<u128>(q[0]) << 64) | q[1];
    const u128 initseq = (static_cast<u128>(q[2]) << 64) | q[3];
    state = 0;
    inc = (initseq << 1) | 1u;
    step();
    state += initstate;
    step();
  }

  uint64_t next64() {
    step();
    const uint64_t x = static_cast<uint64_t>(state >> 64) ^ static_cast<uint64_t>(state);
    const unsigned rot = static_cast<unsigned>(state >> 122);
    return (x >> rot) | (x << ((64u - rot) & 63u));
  }

  double uniform01() { return static_cast<double>(next64() >> 11) * (1.0 / 9007199254740992.0); }
  double uniform(double a, double b) { return a + (b - a) * uniform01(); }
};

enum class Kind { Matrix, Gain, Vector };

struct Param {
  size_t count;
  Kind kind;
  int fan_out, fan_in;
  bool head;
};

// Every parameter in file order (revo.h).
std::vector<Param> param_list(const NetShape& s) {
  std::vector<Param> v;
  auto mat = [&](int out, int in, bool head = false) { v.push_back({static_cast<size_t>(out) * in, Kind::Matrix, out, in, head}); };
  auto vec = [&](int n) { v.push_back({static_cast<size_t>(n), Kind::Vector, 0, 0, false}); };
  auto gain = [&](int n) { v.push_back({static_cast<size_t>(n), Kind::Gain, 0, 0, false}); };
  auto block = [&](int d) {
    gain(d);
    vec(d);
    mat(3 * d, d);
    vec(3 * d);
    mat(d, d);
    vec(d);
    gain(d);
    vec(d);
    mat(s.r * d, d);
    vec(s.r * d);
    mat(d, s.r * d);
    vec(d);
  };
  mat(s.D, s.token_dim());
  vec(s.D);
  for (int i = 0; i < s.L; ++i) block(s.D);
  gain(s.D);
  vec(s.D);
  mat(s.Dd, s.D);
  vec(s.Dd);
  for (int i = 0; i < s.Ld; ++i) block(s.Dd);
  gain(s.Dd);
  vec(s.Dd);
  mat(s.token_dim(), s.Dd, true);
  vec(s.token_dim());
  return v;
}

}  // namespace

void init_weights_random(const NetShape& s, uint64_t seed, float* out) {
  Pcg64 g(seed);
  size_t o = 0;
  for (const Param& p : param_list(s)) {
    if (p.kind == Kind::Matrix) {
      const double b = sqrt(6.0 / static_cast<double>(p.fan_in + p.fan_out));
      for (size_t i = 0; i < p.count; ++i) {
        double w = g.uniform(-b, b);
        if (p.head) w = w * 0.1;
        out[o++] = static_cast<float>(w);
      }
    } else if (p.kind == Kind::Gain) {
      for (size_t i = 0; i < p.count; ++i) out[o++] = static_cast<float>(1.0 + g.uniform(-0.1, 0.1));
    } else {
      for (size_t i = 0; i < p.count; ++i) out[o++] = static_cast<float>(g.uniform(-0.02, 0.02));
    }
  }
}

bool load_weights_file(const char* path, size_t offset_floats, size_t count, float* out, std::string* why) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    *why = std::string("cannot open weights file ") + path;
    return false;
  }
  bool ok = fseek(f, static_cast<long>(offset_floats * sizeof(float)), SEEK_SET) == 0 &&
            fread(out, sizeof(float), count, f) == count;
  if (!ok) *why = std::string("weights file too short: ") + path;
  fclose(f);
  return ok;
}

}  // namespace revo
