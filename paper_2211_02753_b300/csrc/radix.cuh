// Onesweep LSD radix sort of (key, value) pairs (K3); values are uint32 row
// ids or uint64 carried values.
#pragma once

#include "common.cuh"

namespace tdp {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS; // 4096
constexpr int RS_WARPS = RS_THREADS / 32;

inline int radix_passes(int key_bits) { return (key_bits + 7) / 8; }

// Workspace of a sort of up to n pairs with key type of `key_bytes` bytes.
size_t radix_ws_bytes(long long n, int key_bits, int key_bytes, int val_bytes);

// Sorts pairs by the low key_bits bits.  n_max is a host upper bound of the
// element count, d_n (nullable) the actual count on the device.  The result
// lands in keys_out/vals_out; ws holds the ping-pong buffers and scan state.
template <typename K, typename V>
tdp_status radix_sort_pairs(const K *keys_in, const V *vals_in, long long n_max, const long long *d_n,
                            int key_bits, K *keys_out, V *vals_out, void *ws, size_t ws_bytes,
                            int32_t *d_status, cudaStream_t s);

} // namespace tdp
