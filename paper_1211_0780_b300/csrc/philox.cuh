// Counter-based Philox4x32-10 on the device (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.3): ten
// rounds, each multiplying words 0 and 2 by the two Philox constants and
// mixing the high halves into words 1 and 3 with the round key; the key is
// advanced by the two Weyl increments between rounds.  The 64-bit products
// map onto one wide integer multiply-add per word pair on sm_103a.
#pragma once
#include <cstdint>

namespace xy {

struct PhiloxKey {
  uint32_t k0, k1;
};

__device__ __forceinline__ PhiloxKey philox_key(uint64_t seed) {
  return PhiloxKey{static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)};
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const unsigned long long a = static_cast<unsigned long long>(c.x) * 0xD2511F53ull;
    const unsigned long long b = static_cast<unsigned long long>(c.z) * 0xCD9E8D57ull;
    c = make_uint4(static_cast<uint32_t>(b >> 32) ^ c.y ^ k0, static_cast<uint32_t>(b),
                   static_cast<uint32_t>(a >> 32) ^ c.w ^ k1, static_cast<uint32_t>(a));
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The ten round keys of a seed, computed once on the host and passed as a
// kernel parameter: the XOR with the round key then reads its operand from
// the constant bank instead of recomputing the key schedule per call.
struct PhiloxRoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

__host__ __device__ inline PhiloxRoundKeys philox_round_keys(uint64_t seed) {
  PhiloxRoundKeys rk;
  uint32_t a = static_cast<uint32_t>(seed), b = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = a;
    rk.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const unsigned long long a = static_cast<unsigned long long>(c.x) * 0xD2511F53ull;
    const unsigned long long b = static_cast<unsigned long long>(c.z) * 0xCD9E8D57ull;
    c = make_uint4(static_cast<uint32_t>(b >> 32) ^ c.y ^ rk.k0[round], static_cast<uint32_t>(b),
                   static_cast<uint32_t>(a >> 32) ^ c.w ^ rk.k1[round], static_cast<uint32_t>(a));
  }
  return c;
}

// 24-bit uniform in [0, 1); exact in FP32 (and FP64).
__device__ __forceinline__ float u24(uint32_t w) {
  return static_cast<float>(w >> 8) * 5.9604644775390625e-8f;  // 2^-24
}
__device__ __forceinline__ double u24d(uint32_t w) {
  return static_cast<double>(w >> 8) * 5.9604644775390625e-8;
}

}  // namespace xy
