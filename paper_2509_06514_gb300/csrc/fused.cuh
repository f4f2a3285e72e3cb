// fused.cuh — the fused full-domain DPF evaluation + dpXOR kernel for sm_103a.
//
// What one launch computes (§2.3, §3.2, §3.3, Algorithm 1): for every query q of a batch,
//     acc[q] = XOR over j < min(N, 2^m_q) of lsb(R(m_q, j)) * D[j]
// where R is the GGM tree of Eqs. (1)-(3) with AES-128 as the PRF.
//
// How (GB300 mapping of the paper's subtree split and two-stage reduction):
//   * Work unit = (warp tile, query group). A warp tile is 32 * 2^s consecutive leaves: lane l
//     owns the perfect subtree of 2^s leaves rooted at depth m - s (the paper's worker
//     subtrees, §3.2). A query group is up to QC queries of one domain size (§3.4 batching).
//   * The path root -> warp-tile root (the branch-parallel walk, one AES per level) is walked
//     once per query of the group (lane q for query q); the warp then expands the five levels
//     below it for the whole group together, so that every lane holds its subtree root for
//     every query. Each lane expands its subtree depth-first, two children per AES key
//     schedule, and writes the 2^s selection bits of its leaves into shared memory. Selection
//     bits never touch HBM.
//   * The warp then reads the tile's records once (coalesced 16-byte loads, several in flight
//     per lane) and XORs each record into the QC per-query accumulators held in registers
//     (TaskletXOR), folds lanes with warp shuffles (MasterXOR), and XORs the result into the
//     per-query answer in global memory with 64-bit atomic XOR (AggregateSubresults; XOR is
//     order-independent, so the result is bit-exact whatever the order).
//   * MODE 1, the additive answer over Z_2^32: one or two queries per unit, 32-bit shares
//     instead of bits, the queries' walks advanced in turn by chunks of leaves and each chunk's
//     records scanned once for all of them with integer multiply-adds.
//   * A persistent grid, one CTA of 16 or 20 warps per SM: warps take work units from a global
//     counter, units ordered tile-major so that concurrently running warps read the same DB
//     tile (served from L2).
//
// AES: 32-bit T-tables (Te0..Te3) replicated per lane in shared memory. Row x of a 64 KiB
// region holds [Te_a[x] for lanes 0..31 | Te_b[x] for lanes 0..31] (256 bytes), so the byte
// offset of lane L's copy of Te[x] is x*256 + L*4 (+128 for the second table of the region):
// one PRMT builds it from the state word, and the 32 lanes of a warp always hit 32 distinct
// banks. Region A holds Te0|Te1, region B Te2|Te3 (128 KiB). S-box values are read from the
// byte of a T-table entry that equals S[x] (Te2 byte 0, Te3 byte 1, Te0 byte 2, Te1 byte 3).
#pragma once

#include <atomic>
#include <cstdint>

#include "bounds.cuh"
#include "impir_internal.h"

namespace impir {

extern __shared__ __align__(16) uint8_t g_smem[];

// Debug build: n bytes at p lie inside the calling warp's slice of the bit / node / share
// buffer (and inside the launch's dynamic shared memory).
__device__ __forceinline__ bool slice_ok(const void* p, uint32_t n) {
#ifdef IMPIR_BOUNDS
    const long long o = static_cast<const uint8_t*>(p) - g_smem;
    const long long lo = kTableBytes + kSegSmemBytes + (long long)(threadIdx.x >> 5) * s_bctx.warp_slice_bytes;
    return IMPIR_IN_BOUNDS(o >= lo && o + n <= lo + s_bctx.warp_slice_bytes && o + n <= s_bctx.smem_bytes, kSiteBits,
                           o);
#else
    return true;
#endif
}

// A 32-bit word of the warp's bit / share buffer (zero if a debug-build check fails).
__device__ __forceinline__ uint32_t ld_slice(const uint32_t* p) { return slice_ok(p, 4) ? *p : 0u; }

struct Blk {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ Blk bxor(const Blk a, const Blk b) { return {a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w}; }

// Byte offset of lane L's copy of Te[byte b of w]: (byte << 8) | lane4.
__device__ __forceinline__ uint32_t tix(uint32_t w, uint32_t lane4, int b) {
    return __byte_perm(w, lane4, 0x5504u | (uint32_t(b) << 4));
}

template <int K>
__device__ __forceinline__ uint32_t T(uint32_t off) {
    const uint32_t o = off + (K & 1) * 128 + (K >> 1) * 65536;
    if (!IMPIR_IN_BOUNDS(o + 4 <= kTableBytes, kSiteTable, o)) return 0;
    return *reinterpret_cast<const uint32_t*>(g_smem + o);
}

// One full round: SubBytes, ShiftRows, MixColumns, AddRoundKey (FIPS-197 §5.1).
__device__ __forceinline__ Blk aes_round(const Blk s, uint32_t L, uint32_t k0, uint32_t k1, uint32_t k2,
                                         uint32_t k3) {
    Blk o;
    o.x = T<0>(tix(s.x, L, 0)) ^ T<1>(tix(s.y, L, 1)) ^ T<2>(tix(s.z, L, 2)) ^ T<3>(tix(s.w, L, 3)) ^ k0;
    o.y = T<0>(tix(s.y, L, 0)) ^ T<1>(tix(s.z, L, 1)) ^ T<2>(tix(s.w, L, 2)) ^ T<3>(tix(s.x, L, 3)) ^ k1;
    o.z = T<0>(tix(s.z, L, 0)) ^ T<1>(tix(s.w, L, 1)) ^ T<2>(tix(s.x, L, 2)) ^ T<3>(tix(s.y, L, 3)) ^ k2;
    o.w = T<0>(tix(s.w, L, 0)) ^ T<1>(tix(s.x, L, 1)) ^ T<2>(tix(s.y, L, 2)) ^ T<3>(tix(s.z, L, 3)) ^ k3;
    return o;
}

// Final round: SubBytes, ShiftRows, AddRoundKey.
__device__ __forceinline__ Blk aes_final(const Blk s, uint32_t L, uint32_t k0, uint32_t k1, uint32_t k2,
                                         uint32_t k3) {
    Blk o;
    o.x = (T<2>(tix(s.x, L, 0)) & 0xffu) ^ (T<3>(tix(s.y, L, 1)) & 0xff00u) ^ (T<0>(tix(s.z, L, 2)) & 0xff0000u) ^
          (T<1>(tix(s.w, L, 3)) & 0xff000000u) ^ k0;
    o.y = (T<2>(tix(s.y, L, 0)) & 0xffu) ^ (T<3>(tix(s.z, L, 1)) & 0xff00u) ^ (T<0>(tix(s.w, L, 2)) & 0xff0000u) ^
          (T<1>(tix(s.x, L, 3)) & 0xff000000u) ^ k1;
    o.z = (T<2>(tix(s.z, L, 0)) & 0xffu) ^ (T<3>(tix(s.w, L, 1)) & 0xff00u) ^ (T<0>(tix(s.x, L, 2)) & 0xff0000u) ^
          (T<1>(tix(s.y, L, 3)) & 0xff000000u) ^ k2;
    o.w = (T<2>(tix(s.w, L, 0)) & 0xffu) ^ (T<3>(tix(s.x, L, 1)) & 0xff00u) ^ (T<0>(tix(s.y, L, 2)) & 0xff0000u) ^
          (T<1>(tix(s.z, L, 3)) & 0xff000000u) ^ k3;
    return o;
}

// Column 0 of a full round (the only column the leaf bit depends on after round 8).
__device__ __forceinline__ uint32_t aes_round_col0(const Blk s, uint32_t L, uint32_t k0) {
    return T<0>(tix(s.x, L, 0)) ^ T<1>(tix(s.y, L, 1)) ^ T<2>(tix(s.z, L, 2)) ^ T<3>(tix(s.w, L, 3)) ^ k0;
}

// SubWord(RotWord(w)) of the key schedule (FIPS-197 §5.2) on a little-endian word: byte i
// of the result is S[byte i+1 of w]; each lookup's S byte already sits in its target byte
// position, so three byte permutes assemble the word.
__device__ __forceinline__ uint32_t sub_rot(uint32_t w, uint32_t L) {
    const uint32_t lo = __byte_perm(T<2>(tix(w, L, 1)), T<3>(tix(w, L, 2)), 0x0050u);
    const uint32_t hi = __byte_perm(T<0>(tix(w, L, 3)), T<1>(tix(w, L, 0)), 0x7200u);
    return __byte_perm(lo, hi, 0x7610u);
}

// lsb of S[byte 0 of v].
__device__ __forceinline__ uint32_t sbox0_lsb(uint32_t v, uint32_t L) { return T<2>(tix(v, L, 0)) & 1u; }

// Round constants of the key schedule (FIPS-197 §5.2), indexed by round; read from the
// constant cache so the rolled round loops spend no ALU work on them.
__constant__ uint32_t c_rcon[11] = {0x00, 0x01, 0x02, 0x04, 0x08, 0x10, 0x20, 0x40, 0x80, 0x1b, 0x36};

// The round loops below are rolled, or unrolled by two where that measured faster (the node
// pairs and leaf pairs of the keyed PRF: half the loop overhead; -2 % time at 256-byte records):
// the fully unrolled PRF variants overflow the instruction cache of the persistent kernel's hot
// loop, and unrolling by four, or the additive leaf words' loop by two, measured slower.


struct Key4 {
    uint32_t a, b, c, d;
};

__device__ __forceinline__ void ks_next(Key4& k, uint32_t rc, uint32_t L) {
    k.a ^= sub_rot(k.d, L) ^ rc;
    k.b ^= k.a;
    k.c ^= k.b;
    k.d ^= k.c;
}

// ---- keyed PRF: PRF_p(x) = AES-128 with key p over enc(x) = (x, 0, ..., 0) ----

// Round 1 of both encryptions. State after round 0 is p (x = 0) or p ^ 1 (x = 1): they
// differ only in byte 0 of column 0, which only output column 0 of round 1 reads.
__device__ __forceinline__ void keyed_round1(const Blk p, uint32_t L, const Key4& k, Blk& a, Blk& b) {
    const uint32_t c0 = T<1>(tix(p.y, L, 1)) ^ T<2>(tix(p.z, L, 2)) ^ T<3>(tix(p.w, L, 3)) ^ k.a;
    a.x = c0 ^ T<0>(tix(p.x, L, 0));
    b.x = c0 ^ T<0>(tix(p.x ^ 1u, L, 0));
    a.y = T<0>(tix(p.y, L, 0)) ^ T<1>(tix(p.z, L, 1)) ^ T<2>(tix(p.w, L, 2)) ^ T<3>(tix(p.x, L, 3)) ^ k.b;
    a.z = T<0>(tix(p.z, L, 0)) ^ T<1>(tix(p.w, L, 1)) ^ T<2>(tix(p.x, L, 2)) ^ T<3>(tix(p.y, L, 3)) ^ k.c;
    a.w = T<0>(tix(p.w, L, 0)) ^ T<1>(tix(p.x, L, 1)) ^ T<2>(tix(p.y, L, 2)) ^ T<3>(tix(p.z, L, 3)) ^ k.d;
    b.y = a.y;
    b.z = a.z;
    b.w = a.w;
}

// Both children of parent seed p: PRF_p(0) ^ ca and PRF_p(1) ^ cb (the correction words
// are folded into the last AddRoundKey).
__device__ __forceinline__ void keyed_pair(const Blk p, uint32_t L, const Blk ca, const Blk cb, Blk& a, Blk& b) {
    Key4 k{p.x, p.y, p.z, p.w};
    ks_next(k, 0x01u, L);
    keyed_round1(p, L, k, a, b);
#pragma unroll 2
    for (int r = 2; r <= 9; ++r) {
        ks_next(k, c_rcon[r], L);
        a = aes_round(a, L, k.a, k.b, k.c, k.d);
        b = aes_round(b, L, k.a, k.b, k.c, k.d);
    }
    ks_next(k, 0x36u, L);
    a = aes_final(a, L, k.a ^ ca.x, k.b ^ ca.y, k.c ^ ca.z, k.d ^ ca.w);
    b = aes_final(b, L, k.a ^ cb.x, k.b ^ cb.y, k.c ^ cb.z, k.d ^ cb.w);
}

// lsb of both PRF outputs: rounds 1-8 in full, then only what byte 0 of the output needs:
// column 0 of round 9 and byte 0 of round 10 (whose round-key byte 0 is
// rk9.w0.b0 ^ S[rk9.w3.b1] ^ 0x36).
__device__ __forceinline__ uint32_t keyed_leaf_bits(const Blk p, uint32_t L) {
    Key4 k{p.x, p.y, p.z, p.w};
    Blk a, b;
    ks_next(k, 0x01u, L);
    keyed_round1(p, L, k, a, b);
    ks_next(k, 0x02u, L);
    a = aes_round(a, L, k.a, k.b, k.c, k.d);
    b = aes_round(b, L, k.a, k.b, k.c, k.d);
#pragma unroll 2
    for (int r = 3; r <= 8; ++r) {
        ks_next(k, c_rcon[r], L);
        a = aes_round(a, L, k.a, k.b, k.c, k.d);
        b = aes_round(b, L, k.a, k.b, k.c, k.d);
    }
    ks_next(k, 0x1bu, L);
    const uint32_t a9 = aes_round_col0(a, L, k.a);
    const uint32_t b9 = aes_round_col0(b, L, k.a);
    const uint32_t kbit = (k.a ^ sbox0_lsb(k.d >> 8, L)) & 1u;  // lsb(0x36) = 0
    return ((sbox0_lsb(a9, L) ^ kbit) & 1u) | (((sbox0_lsb(b9, L) ^ kbit) & 1u) << 1);
}

// One child's PRF output (the root-to-subtree walk): x may differ between lanes.
__device__ __forceinline__ Blk keyed_one(const Blk p, uint32_t x, uint32_t L) {
    Key4 k{p.x, p.y, p.z, p.w};
    Blk s{p.x ^ x, p.y, p.z, p.w};
#pragma unroll 1
    for (int r = 1; r <= 9; ++r) {
        ks_next(k, c_rcon[r], L);
        s = aes_round(s, L, k.a, k.b, k.c, k.d);
    }
    ks_next(k, 0x36u, L);
    return aes_final(s, L, k.a, k.b, k.c, k.d);
}

// Word 0 (output bytes 0..3) of both PRF outputs: rounds 1-9 in full, then only column 0
// of round 10 (the additive answer's shares are the leaves' low 32 bits).
__device__ __forceinline__ void keyed_leaf_words(const Blk p, uint32_t L, uint32_t& wa, uint32_t& wb) {
    Key4 k{p.x, p.y, p.z, p.w};
    Blk a, b;
    ks_next(k, 0x01u, L);
    keyed_round1(p, L, k, a, b);
#pragma unroll 1
    for (int r = 2; r <= 9; ++r) {
        ks_next(k, c_rcon[r], L);
        a = aes_round(a, L, k.a, k.b, k.c, k.d);
        b = aes_round(b, L, k.a, k.b, k.c, k.d);
    }
    const uint32_t k10 = k.a ^ sub_rot(k.d, L) ^ 0x36u;
    wa = (T<2>(tix(a.x, L, 0)) & 0xffu) ^ (T<3>(tix(a.y, L, 1)) & 0xff00u) ^ (T<0>(tix(a.z, L, 2)) & 0xff0000u) ^
         (T<1>(tix(a.w, L, 3)) & 0xff000000u) ^ k10;
    wb = (T<2>(tix(b.x, L, 0)) & 0xffu) ^ (T<3>(tix(b.y, L, 1)) & 0xff00u) ^ (T<0>(tix(b.z, L, 2)) & 0xff0000u) ^
         (T<1>(tix(b.w, L, 3)) & 0xff000000u) ^ k10;
}

// ---- MMO PRF: PRF_p(x) = AES_{K_x}(p) ^ p with fixed round keys rk[x][44] ----

__device__ __forceinline__ void mmo_pair(const Blk p, uint32_t L, const uint32_t (&rk)[2][44], const Blk ca,
                                         const Blk cb, Blk& a, Blk& b) {
    a = {p.x ^ rk[0][0], p.y ^ rk[0][1], p.z ^ rk[0][2], p.w ^ rk[0][3]};
    b = {p.x ^ rk[1][0], p.y ^ rk[1][1], p.z ^ rk[1][2], p.w ^ rk[1][3]};
#pragma unroll 1
    for (int r = 1; r <= 9; ++r) {
        a = aes_round(a, L, rk[0][4 * r], rk[0][4 * r + 1], rk[0][4 * r + 2], rk[0][4 * r + 3]);
        b = aes_round(b, L, rk[1][4 * r], rk[1][4 * r + 1], rk[1][4 * r + 2], rk[1][4 * r + 3]);
    }
    const Blk pa = bxor(p, ca), pb = bxor(p, cb);
    a = aes_final(a, L, rk[0][40] ^ pa.x, rk[0][41] ^ pa.y, rk[0][42] ^ pa.z, rk[0][43] ^ pa.w);
    b = aes_final(b, L, rk[1][40] ^ pb.x, rk[1][41] ^ pb.y, rk[1][42] ^ pb.z, rk[1][43] ^ pb.w);
}

__device__ __forceinline__ uint32_t mmo_leaf_bits(const Blk p, uint32_t L, const uint32_t (&rk)[2][44]) {
    Blk a = {p.x ^ rk[0][0], p.y ^ rk[0][1], p.z ^ rk[0][2], p.w ^ rk[0][3]};
    Blk b = {p.x ^ rk[1][0], p.y ^ rk[1][1], p.z ^ rk[1][2], p.w ^ rk[1][3]};
#pragma unroll 1
    for (int r = 1; r <= 8; ++r) {
        a = aes_round(a, L, rk[0][4 * r], rk[0][4 * r + 1], rk[0][4 * r + 2], rk[0][4 * r + 3]);
        b = aes_round(b, L, rk[1][4 * r], rk[1][4 * r + 1], rk[1][4 * r + 2], rk[1][4 * r + 3]);
    }
    const uint32_t a9 = aes_round_col0(a, L, rk[0][36]);
    const uint32_t b9 = aes_round_col0(b, L, rk[1][36]);
    const uint32_t ba = (sbox0_lsb(a9, L) ^ rk[0][40] ^ p.x) & 1u;
    const uint32_t bb = (sbox0_lsb(b9, L) ^ rk[1][40] ^ p.x) & 1u;
    return ba | (bb << 1);
}

__device__ __forceinline__ void mmo_leaf_words(const Blk p, uint32_t L, const uint32_t (&rk)[2][44], uint32_t& wa,
                                               uint32_t& wb) {
    Blk a = {p.x ^ rk[0][0], p.y ^ rk[0][1], p.z ^ rk[0][2], p.w ^ rk[0][3]};
    Blk b = {p.x ^ rk[1][0], p.y ^ rk[1][1], p.z ^ rk[1][2], p.w ^ rk[1][3]};
#pragma unroll 1
    for (int r = 1; r <= 9; ++r) {
        a = aes_round(a, L, rk[0][4 * r], rk[0][4 * r + 1], rk[0][4 * r + 2], rk[0][4 * r + 3]);
        b = aes_round(b, L, rk[1][4 * r], rk[1][4 * r + 1], rk[1][4 * r + 2], rk[1][4 * r + 3]);
    }
    wa = (T<2>(tix(a.x, L, 0)) & 0xffu) ^ (T<3>(tix(a.y, L, 1)) & 0xff00u) ^ (T<0>(tix(a.z, L, 2)) & 0xff0000u) ^
         (T<1>(tix(a.w, L, 3)) & 0xff000000u) ^ rk[0][40] ^ p.x;
    wb = (T<2>(tix(b.x, L, 0)) & 0xffu) ^ (T<3>(tix(b.y, L, 1)) & 0xff00u) ^ (T<0>(tix(b.z, L, 2)) & 0xff0000u) ^
         (T<1>(tix(b.w, L, 3)) & 0xff000000u) ^ rk[1][40] ^ p.x;
}

__device__ __forceinline__ Blk mmo_one(const Blk p, uint32_t x, uint32_t L, const uint32_t (&rk)[2][44]) {
    Blk s = {p.x ^ (x ? rk[1][0] : rk[0][0]), p.y ^ (x ? rk[1][1] : rk[0][1]), p.z ^ (x ? rk[1][2] : rk[0][2]),
             p.w ^ (x ? rk[1][3] : rk[0][3])};
#pragma unroll 1
    for (int r = 1; r <= 9; ++r)
        s = aes_round(s, L, x ? rk[1][4 * r] : rk[0][4 * r], x ? rk[1][4 * r + 1] : rk[0][4 * r + 1],
                      x ? rk[1][4 * r + 2] : rk[0][4 * r + 2], x ? rk[1][4 * r + 3] : rk[0][4 * r + 3]);
    s = aes_final(s, L, x ? rk[1][40] : rk[0][40], x ? rk[1][41] : rk[0][41], x ? rk[1][42] : rk[0][42],
                  x ? rk[1][43] : rk[0][43]);
    return bxor(s, p);
}

// ---- codewords C_t[x][d] of a wire key (8-byte aligned entries) ----

__device__ __forceinline__ size_t cw_off(uint32_t m, uint32_t t, uint32_t x, uint32_t d) {
    return 8 + size_t(t) * 32 * (m + 1) + (size_t(x) * (m + 1) + d) * 16;
}

// Debug build: the n bytes at kq + off lie inside the key (domain bits m) and, when the key
// buffer's size is known, inside the buffer.
__device__ __forceinline__ bool key_bytes_ok(const uint8_t* kq, uint32_t m, size_t off, uint32_t n) {
#ifdef IMPIR_BOUNDS
    const long long rel = (kq - s_bctx.keys) + (long long)off;
    const bool in_key = off + n <= 8 + 64ull * (m + 1);
    const bool in_buf = rel >= 0 && (s_bctx.keys_bytes == 0 || (unsigned long long)rel + n <= s_bctx.keys_bytes);
    return IMPIR_IN_BOUNDS(in_key && in_buf, kSiteKey, rel);
#else
    return true;
#endif
}

__device__ __forceinline__ Blk cw_load(const uint8_t* kq, uint32_t m, uint32_t t, uint32_t x, uint32_t d) {
    const size_t off = cw_off(m, t, x, d);
    if (!key_bytes_ok(kq, m, off, 16)) return {0, 0, 0, 0};
    const uint2* p = reinterpret_cast<const uint2*>(kq + off);
    const uint2 lo = __ldg(p), hi = __ldg(p + 1);
    return {lo.x, lo.y, hi.x, hi.y};
}

__device__ __forceinline__ uint32_t cw_lsb(const uint8_t* kq, uint32_t m, uint32_t t, uint32_t x, uint32_t d) {
    const size_t off = cw_off(m, t, x, d);
    if (!key_bytes_ok(kq, m, off, 1)) return 0;
    return __ldg(kq + off) & 1u;
}

// A 16-byte database word (debug build: inside the words the launch may read, else zero).
__device__ __forceinline__ uint4 ld_db(const uint4* p) {
#ifdef IMPIR_BOUNDS
    const long long w = p - s_bctx.db;
    if (!IMPIR_IN_BOUNDS(w >= 0 && (unsigned long long)w < s_bctx.db_words, kSiteRecord, w)) return make_uint4(0, 0, 0, 0);
#endif
    return __ldg(p);
}

// Index of the q-th query of a group whose sorted query indices start at qidx (debug build:
// the position lies inside the sorted permutation and the index names a query of the batch).
__device__ __forceinline__ uint32_t query_at(const FusedParams& P, const uint32_t* qidx, uint32_t q) {
#ifdef IMPIR_BOUNDS
    const long long i = (qidx - reinterpret_cast<const uint32_t*>(P.ws + P.lay.off_perm)) + (long long)q;
    if (!IMPIR_IN_BOUNDS(i >= 0 && i < (long long)P.n_queries, kSiteQuery, i)) return 0;
    const uint32_t v = qidx[q];
    if (!IMPIR_IN_BOUNDS(v < P.n_queries, kSiteQuery, v)) return 0;
    return v;
#else
    return qidx[q];
#endif
}

// The wire key of query qi (debug build: its header lies inside the key buffer when the size
// of that is known).
__device__ __forceinline__ const uint8_t* query_key(const FusedParams& P, uint32_t qi) {
    const uint32_t off = P.key_off[qi];
    if (!IMPIR_IN_BOUNDS(P.keys_bytes == 0 || off + 8ull <= P.keys_bytes, kSiteKey, off)) return P.keys;
    return P.keys + off;
}

__device__ __forceinline__ void mad4(uint4& a, const uint4 v, uint32_t s) {
    a.x += v.x * s;
    a.y += v.y * s;
    a.z += v.z * s;
    a.w += v.w * s;
}

__device__ __forceinline__ uint4 add4(const uint4 a, const uint4 b) {
    return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ void red_add(uint4* dst, const uint4 v) {
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    if (v.x) atomicAdd(d, v.x);
    if (v.y) atomicAdd(d + 1, v.y);
    if (v.z) atomicAdd(d + 2, v.z);
    if (v.w) atomicAdd(d + 3, v.w);
}

// Adds v into word k of query qi's accumulator (debug build: both inside the batch's answers).
__device__ __forceinline__ void acc_add(const FusedParams& P, uint4* acc_out, uint32_t qi, uint32_t k, const uint4 v) {
    if (!IMPIR_IN_BOUNDS(qi < P.n_queries && k < P.words, kSiteAcc, (unsigned long long)qi * P.words + k)) return;
    red_add(acc_out + size_t(qi) * P.words + k, v);
}

// Additive answer of one chunk of a warp tile for the unit's queries: acc_q += share_q * D[r],
// word by word mod 2^32 (records read as little-endian 32-bit words), added into each query's
// accumulator; every record is loaded once for all the queries. The chunk holds `runs` runs of
// `run_len` consecutive records; run l starts at tile record (l << sq) + chunk_off and query
// q's shares of it sit at vals[q * qstride + l * run_len ...]. Records at or past `nrec` (the
// DB end) are skipped; runs start in ascending order.
template <int QC, int NK>
__device__ __forceinline__ void scan_chunk_add(const FusedParams& P, uint64_t tile_base, uint32_t nrec,
                                               const uint32_t* vals, uint32_t qstride, uint32_t count,
                                               const uint32_t* qidx, uint32_t runs, uint32_t run_len, uint32_t sq,
                                               uint32_t chunk_off, uint4* acc_out, uint32_t lane) {
    const uint32_t W = P.words;
    const uint4* tile = P.db + (tile_base - P.rec_lo) * W;
    if constexpr (NK == 1) {
        // W <= 32: R records per step, lane -> (record lr, word lk)
        const uint32_t R = 32u / W, lr = lane / W, lk = lane - lr * W;
        const bool on = lr < R;
        uint4 acc[QC];
#pragma unroll
        for (int q = 0; q < QC; ++q) acc[q] = make_uint4(0, 0, 0, 0);
        constexpr int RB = QC == 1 ? 8 : 4;  // records' loads in flight per lane (fewer with more accumulators)
        for (uint32_t l = 0; l < runs; ++l) {
            const uint32_t rb = (l << sq) + chunk_off;
            if (rb >= nrec) break;
            const uint32_t n = min(run_len, nrec - rb);
            const uint32_t* vl = vals + l * run_len;
            const uint4* bl = tile + size_t(rb) * W + lk;
            for (uint32_t r0 = 0; r0 < n; r0 += RB * R) {
                uint4 v[RB];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const uint32_t r = r0 + u * R + lr;
                    v[u] = (on && r < n) ? ld_db(bl + size_t(r) * W) : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const uint32_t r = r0 + u * R + lr;
                    if (on && r < n)
#pragma unroll
                        for (int q = 0; q < QC; ++q)
                            if (uint32_t(q) < count) mad4(acc[q], v[u], ld_slice(&vl[q * qstride + r]));
                }
            }
        }
        if (R * W == 32) {
            for (uint32_t off = W; off < 32; off <<= 1)
#pragma unroll
                for (int q = 0; q < QC; ++q)
                    acc[q] = add4(acc[q], make_uint4(__shfl_xor_sync(0xffffffffu, acc[q].x, off),
                                                     __shfl_xor_sync(0xffffffffu, acc[q].y, off),
                                                     __shfl_xor_sync(0xffffffffu, acc[q].z, off),
                                                     __shfl_xor_sync(0xffffffffu, acc[q].w, off)));
            if (lr == 0)
#pragma unroll
                for (int q = 0; q < QC; ++q)
                    if (uint32_t(q) < count) acc_add(P, acc_out, query_at(P, qidx, q), lk, acc[q]);
        } else if (on) {
#pragma unroll
            for (int q = 0; q < QC; ++q)
                if (uint32_t(q) < count) acc_add(P, acc_out, query_at(P, qidx, q), lk, acc[q]);
        }
    } else {
        // W > 32: the whole warp reads one record per step, NK words per lane, in column passes
        for (uint32_t k0 = 0; k0 < W; k0 += 32 * NK) {
            uint4 acc[QC][NK];
#pragma unroll
            for (int q = 0; q < QC; ++q)
#pragma unroll
                for (int c = 0; c < NK; ++c) acc[q][c] = make_uint4(0, 0, 0, 0);
            for (uint32_t l = 0; l < runs; ++l) {
                const uint32_t rb = (l << sq) + chunk_off;
                if (rb >= nrec) break;
                const uint32_t n = min(run_len, nrec - rb);
                const uint32_t* vl = vals + l * run_len;
#pragma unroll 4
                for (uint32_t r = 0; r < n; ++r) {
                    const uint4* rec = tile + size_t(rb + r) * W;
                    uint4 v[NK];
#pragma unroll
                    for (int c = 0; c < NK; ++c) {
                        const uint32_t k = k0 + lane + 32 * c;
                        v[c] = k < W ? ld_db(rec + k) : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int q = 0; q < QC; ++q)
                        if (uint32_t(q) < count) {
                            const uint32_t sv = ld_slice(&vl[q * qstride + r]);
#pragma unroll
                            for (int c = 0; c < NK; ++c) mad4(acc[q][c], v[c], sv);
                        }
                }
            }
#pragma unroll
            for (int q = 0; q < QC; ++q)
                if (uint32_t(q) < count)
#pragma unroll
                    for (int c = 0; c < NK; ++c) {
                        const uint32_t k = k0 + lane + 32 * c;
                        if (k < W) acc_add(P, acc_out, query_at(P, qidx, q), k, acc[q][c]);
                    }
        }
    }
}

// Selection bits of lane's subtree: root -> depth D walk (Eq. (3) one edge per level), then
// a depth-first expansion down to the leaves at depth m; bit r of `bits` (relative to the
// warp tile) is lsb(R(m, tile_first_leaf + r)).
// The walk starts from `start`, the node at depth d0 on the lane's path (the root with d0 = 0,
// or the warp-tile root the warp computed once for this query).
template <int PRF>
__device__ __forceinline__ Blk walk_down(const FusedParams& P, const uint8_t* kq, uint32_t m, uint32_t D, uint64_t sub,
                                         uint32_t L, const Blk start, uint32_t d0) {
    Blk node = start;
    for (uint32_t d = d0 + 1; d <= D; ++d) {
        const uint32_t x = uint32_t(sub >> (D - d)) & 1u;
        const uint32_t t = node.x & 1u;
        const Blk c = cw_load(kq, m, t, x, d);
        const Blk f = PRF == 0 ? keyed_one(node, x, L) : mmo_one(node, x, L, P.mmo_rk);
        node = bxor(f, c);
    }
    return node;
}

template <int PRF>
__device__ __forceinline__ void lane_eval(const FusedParams& P, const uint8_t* kq, uint32_t m, uint32_t D,
                                          uint64_t sub, uint32_t sq, uint32_t* bits, uint32_t lane, uint32_t L,
                                          const Blk start, uint32_t d0) {
    Blk node = walk_down<PRF>(P, kq, m, D, sub, L, start, d0);
    if (sq == 0) {
        if (slice_ok(&bits[lane >> 5], 4)) atomicOr(&bits[lane >> 5], (node.x & 1u) << (lane & 31));
        return;
    }
    Blk stk[kMaxLaneBits];
    uint32_t depth = D, p = 0, acc = 0;
    const uint32_t npairs = 1u << (sq - 1);
    for (;;) {
        const uint32_t t = node.x & 1u;
        if (depth == m - 1) {
            uint32_t b2 = PRF == 0 ? keyed_leaf_bits(node, L) : mmo_leaf_bits(node, L, P.mmo_rk);
            b2 ^= cw_lsb(kq, m, t, 0, m) | (cw_lsb(kq, m, t, 1, m) << 1);
            acc |= b2 << ((2 * p) & 31);
            ++p;
            if (sq >= 5 && (p & 15) == 0) {
                uint32_t* w = &bits[(lane << (sq - 5)) + ((p - 1) >> 4)];
                if (slice_ok(w, 4)) *w = acc;
                acc = 0;
            }
            if (p == npairs) break;
            depth = m - 1 - (__ffs(int(p)) - 1);
            if (IMPIR_IN_BOUNDS(depth - D < kMaxLaneBits, kSiteStack, depth - D)) node = stk[depth - D];
        } else {
            const Blk c0 = cw_load(kq, m, t, 0, depth + 1);
            const Blk c1 = cw_load(kq, m, t, 1, depth + 1);
            Blk a, b;
            if (PRF == 0)
                keyed_pair(node, L, c0, c1, a, b);
            else
                mmo_pair(node, L, P.mmo_rk, c0, c1, a, b);
            ++depth;
            if (IMPIR_IN_BOUNDS(depth - D < kMaxLaneBits, kSiteStack, depth - D)) stk[depth - D] = b;
            node = a;
        }
    }
    if (sq < 5 && slice_ok(&bits[(lane << sq) >> 5], 4)) atomicOr(&bits[(lane << sq) >> 5], acc << ((lane << sq) & 31));
}

// ---- additive answer (MODE 1) ----

// A lane's depth-first walk of one query's subtree, resumable after every chunk of leaves so
// that the warp can advance several queries' walks between two scans.
struct AddWalk {
    Blk node;               // the next node to expand
    uint32_t depth, p;      // its depth; leaf pairs written so far
    Blk stk[kMaxLaneBits];  // pending right children, by depth - D
};

// Advances the walk by ch leaves (ch >= 2, even): the shares (-1)^party low32(R(m, j)) of the
// lane's next ch leaves go to shares[lane * ch + 0 .. ch - 1].
template <int PRF>
__device__ __forceinline__ void add_walk_chunk(const FusedParams& P, const uint8_t* kq, uint32_t m, uint32_t D,
                                               uint32_t sq, AddWalk& w, uint32_t ch, uint32_t* shares, uint32_t lane,
                                               uint32_t L, uint32_t neg) {
    Blk node = w.node;
    uint32_t depth = w.depth, p = w.p;
    const uint32_t npairs = 1u << (sq - 1), end = p + ch / 2;
    for (;;) {
        const uint32_t t = node.x & 1u;
        if (depth == m - 1) {
            uint32_t wa, wb;
            if (PRF == 0)
                keyed_leaf_words(node, L, wa, wb);
            else
                mmo_leaf_words(node, L, P.mmo_rk, wa, wb);
            wa ^= cw_load(kq, m, t, 0, m).x;
            wb ^= cw_load(kq, m, t, 1, m).x;
            const uint32_t r = lane * ch + ((2 * p) & (ch - 1));
            if (slice_ok(&shares[r], 8)) {
                shares[r] = (wa ^ neg) - neg;
                shares[r + 1] = (wb ^ neg) - neg;
            }
            ++p;
            if (p == npairs) break;
            depth = m - 1 - (__ffs(int(p)) - 1);
            if (IMPIR_IN_BOUNDS(depth - D < kMaxLaneBits, kSiteStack, depth - D)) node = w.stk[depth - D];
            if (p == end) break;
        } else {
            const Blk c0 = cw_load(kq, m, t, 0, depth + 1);
            const Blk c1 = cw_load(kq, m, t, 1, depth + 1);
            Blk a, b;
            if (PRF == 0)
                keyed_pair(node, L, c0, c1, a, b);
            else
                mmo_pair(node, L, P.mmo_rk, c0, c1, a, b);
            ++depth;
            if (IMPIR_IN_BOUNDS(depth - D < kMaxLaneBits, kSiteStack, depth - D)) w.stk[depth - D] = b;
            node = a;
        }
    }
    w.node = node;
    w.depth = depth;
    w.p = p;
}

// One work unit of the additive answer: the group's queries over one warp tile. Every lane
// walks from the warp-tile root (`top`, held by lane q for query q) to its subtree root for
// each query, then the warp alternates: each query's walk advances by one chunk of ch leaves
// per lane (ch = 32 / QC, so the group's shares fill 4 KiB per warp), and the chunk's records
// are scanned once for all the queries. Lanes past the DB end walk nodes that exist in the
// tree; the scan skips their records. All 32 lanes take part (the scan is warp-wide).
template <int QC, int NK>
__device__ __forceinline__ void unit_add(const FusedParams& P, const GroupDesc& gd, const uint32_t* qidx,
                                         uint64_t tile_base, uint32_t nrec, uint64_t sub, uint32_t sq, uint32_t D,
                                         uint32_t Dt, const Blk top, uint32_t* shares, uint4* acc_out, uint32_t lane,
                                         uint32_t L) {
    const uint32_t m = gd.m, count = gd.count;
    AddWalk w[QC];
    uint32_t neg[QC];
    const uint32_t ch = sq == 0 ? 1u : min(1u << sq, 32u / QC), qstride = 32 * ch;
#pragma unroll
    for (int q = 0; q < QC; ++q) {
        neg[q] = 0;
        if (uint32_t(q) < count) {
            const uint8_t* kq = query_key(P, query_at(P, qidx, q));
            const Blk start{__shfl_sync(0xffffffffu, top.x, q), __shfl_sync(0xffffffffu, top.y, q),
                            __shfl_sync(0xffffffffu, top.z, q), __shfl_sync(0xffffffffu, top.w, q)};
            w[q].node = kq[1] == 0 ? walk_down<0>(P, kq, m, D, sub, L, start, Dt)
                                   : walk_down<1>(P, kq, m, D, sub, L, start, Dt);
            w[q].depth = D;
            w[q].p = 0;
            neg[q] = kq[3] ? 0xffffffffu : 0u;  // party 1 negates its shares (mod 2^32)
        }
    }
    if (sq == 0) {  // one leaf per lane: the subtree root is the leaf
#pragma unroll
        for (int q = 0; q < QC; ++q)
            if (uint32_t(q) < count && slice_ok(&shares[q * qstride + lane], 4))
                shares[q * qstride + lane] = (w[q].node.x ^ neg[q]) - neg[q];
        __syncwarp();
        scan_chunk_add<QC, NK>(P, tile_base, nrec, shares, qstride, count, qidx, 1, 32, 0, 0, acc_out, lane);
        return;
    }
    // with lane subtrees of at most ch leaves the chunk is the whole tile (one run of
    // consecutive records), else 32 runs of ch records
    const uint32_t runs = (1u << sq) > ch ? 32u : 1u, run_len = runs == 32 ? ch : (32u << sq);
    const uint32_t nchunks = (1u << sq) / ch;
    for (uint32_t c = 0; c < nchunks; ++c) {
#pragma unroll
        for (int q = 0; q < QC; ++q)
            if (uint32_t(q) < count) {
                const uint8_t* kq = query_key(P, query_at(P, qidx, q));
                if (kq[1] == 0)
                    add_walk_chunk<0>(P, kq, m, D, sq, w[q], ch, shares + q * qstride, lane, L, neg[q]);
                else
                    add_walk_chunk<1>(P, kq, m, D, sq, w[q], ch, shares + q * qstride, lane, L, neg[q]);
            }
        __syncwarp();
        scan_chunk_add<QC, NK>(P, tile_base, nrec, shares, qstride, count, qidx, runs, run_len, sq, c * ch, acc_out,
                               lane);
        __syncwarp();
    }
}

__device__ __forceinline__ void red_xor(uint4* dst, const uint4 v) {
    if (v.x | v.y)
        atomicXor(reinterpret_cast<unsigned long long*>(dst),
                  (unsigned long long)v.x | ((unsigned long long)v.y << 32));
    if (v.z | v.w)
        atomicXor(reinterpret_cast<unsigned long long*>(dst) + 1,
                  (unsigned long long)v.z | ((unsigned long long)v.w << 32));
}

// XORs v into word k of query qi's accumulator (debug build: both inside the batch's answers).
__device__ __forceinline__ void acc_xor(const FusedParams& P, uint4* acc_out, uint32_t qi, uint32_t k, const uint4 v) {
    if (!IMPIR_IN_BOUNDS(qi < P.n_queries && k < P.words, kSiteAcc, (unsigned long long)qi * P.words + k)) return;
    red_xor(acc_out + size_t(qi) * P.words + k, v);
}

// All-ones if bit 31 of x is set, else zero, as the high word of the signed product x * one
// (one == 1 at run time): an integer multiply (FMA pipe) instead of an arithmetic shift (ALU pipe).
__device__ __forceinline__ uint32_t sign_mask_fma(uint32_t x, uint32_t one) {
    uint32_t m;
    asm("mul.hi.s32 %0, %1, %2;" : "=r"(m) : "r"(x), "r"(one));
    return m;
}

__device__ __forceinline__ uint4 bxor3(const uint4 a, const uint4 b, const uint4 c) {
    return make_uint4(a.x ^ b.x ^ c.x, a.y ^ b.y ^ c.y, a.z ^ b.z ^ c.z, a.w ^ b.w ^ c.w);
}

__device__ __forceinline__ void xor_masked(uint4& a, const uint4 v, uint32_t msk) {
    a.x ^= v.x & msk;
    a.y ^= v.y & msk;
    a.z ^= v.z & msk;
    a.w ^= v.w & msk;
}

__device__ __forceinline__ uint4 bxor4(const uint4 a, const uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

__device__ __forceinline__ uint4 shfl_xor4(const uint4 v, int off) {
    return make_uint4(__shfl_xor_sync(0xffffffffu, v.x, off), __shfl_xor_sync(0xffffffffu, v.y, off),
                      __shfl_xor_sync(0xffffffffu, v.z, off), __shfl_xor_sync(0xffffffffu, v.w, off));
}

// dpXOR of one warp tile for the group's queries: records [tile_base, tile_base + nrec).
// Selection bits are read one 32-bit word (32 records) per query at a time.
template <int QC, int NK>
__device__ __forceinline__ void scan_tile(const FusedParams& P, uint64_t tile_base, uint32_t nrec,
                                          const uint32_t* bits, uint32_t count, const uint32_t* qidx, uint4* acc_out,
                                          uint32_t lane) {
    const uint32_t W = P.words;
    const uint32_t bw = P.bits_words;
    if constexpr (NK == 1) {
        // W <= 32: R records per step, lane -> (record lr, word lk)
        const uint32_t R = 32u / W, lr = lane / W, lk = lane - lr * W;
        const bool on = lr < R;
        // 1 << R, from a value the compiler cannot see through, so that multiplying by it stays an
        // integer multiply-add (FMA pipe) instead of becoming a shift (ALU pipe, which the AES
        // engine keeps busy)
        const uint32_t stepmul = (P.n_queries != 0 ? 1u : 0u) << R;
        uint4 acc[QC];
#pragma unroll
        for (int q = 0; q < QC; ++q) acc[q] = make_uint4(0, 0, 0, 0);
        const uint4* base = P.db + (tile_base - P.rec_lo) * W + lk;
        for (uint32_t c0 = 0; c0 < nrec; c0 += 32) {
            uint32_t sel[QC];
#pragma unroll
            for (int q = 0; q < QC; ++q) sel[q] = ld_slice(&bits[q * bw + (c0 >> 5)]) >> lr;  // bit i*R: record c0+i*R+lr
            const uint32_t nloc = min(32u, nrec - c0);
            if (R == 1) {
                // one record per step for the whole warp: its selection bits are warp-uniform;
                // four records' loads in flight, one bit mask per record shared by the queries
                for (uint32_t i0 = 0; i0 < nloc; i0 += 4) {
                    uint4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = (on && i0 + u < nloc) ? ld_db(base + size_t(c0 + i0 + u) * W) : make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t bm = 1u << (i0 + u);
#pragma unroll
                        for (int q = 0; q < QC; ++q)
                            if (sel[q] & bm) acc[q] = bxor4(acc[q], v[u]);
                    }
                }
            } else {
                // bit-reversed selection words: step i's bit sits in bit 31 of sh << i, so a step
                // takes one arithmetic shift for the mask and one multiply by 2^R to advance
                uint32_t sh[QC];
#pragma unroll
                for (int q = 0; q < QC; ++q) sh[q] = __brev(sel[q]);
                // four steps' loads in flight before their XORs
                for (uint32_t i0 = 0; i0 < 32; i0 += 4 * R) {
                    uint4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t i = i0 + u * R;
                        v[u] = (on && i < 32 && i + lr < nloc) ? ld_db(base + size_t(c0 + i + lr) * W)
                                                               : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int q = 0; q < QC; ++q) {
                            xor_masked(acc[q], v[u], uint32_t(int32_t(sh[q]) >> 31));
                            asm("mul.lo.u32 %0, %0, %1;" : "+r"(sh[q]) : "r"(stepmul));
                        }
                }
            }
        }
        if (R * W == 32) {
            for (uint32_t off = W; off < 32; off <<= 1)
#pragma unroll
                for (int q = 0; q < QC; ++q) acc[q] = bxor4(acc[q], shfl_xor4(acc[q], int(off)));
            if (lr == 0)
#pragma unroll
                for (int q = 0; q < QC; ++q)
                    if (uint32_t(q) < count) acc_xor(P, acc_out, query_at(P, qidx, q), lk, acc[q]);
        } else if (on) {
#pragma unroll
            for (int q = 0; q < QC; ++q)
                if (uint32_t(q) < count) acc_xor(P, acc_out, query_at(P, qidx, q), lk, acc[q]);
        }
    } else {
        // W > 32: the whole warp reads one record per step, NK words per lane, in column
        // passes; a record's selection bits are warp-uniform. The compiler predicates a
        // conditional XOR of this size rather than branching (and real branches measured slower),
        // so every query costs ALU work on every record either way. With NK = 2 the XOR is masked,
        // the mask taken on the FMA pipe; with NK >= 4 two records are taken together, both selected
        // costing one 3-input XOR.
        const uint32_t one = P.n_queries != 0 ? 1u : 0u;  // 1, opaque to the compiler
        constexpr int RB = NK <= 2 ? 4 : NK == 4 ? 2 : 1;  // records' loads in flight per lane
        for (uint32_t k0 = 0; k0 < W; k0 += 32 * NK) {
            uint4 acc[QC][NK];
#pragma unroll
            for (int q = 0; q < QC; ++q)
#pragma unroll
                for (int c = 0; c < NK; ++c) acc[q][c] = make_uint4(0, 0, 0, 0);
            // this lane's words of the tile's records in this pass: record r, column c at
            // tb + r * W + 32 * c
            const uint4* tb = P.db + (tile_base - P.rec_lo) * W + k0 + lane;
            bool kon[NK];
#pragma unroll
            for (int c = 0; c < NK; ++c) kon[c] = k0 + lane + 32 * c < W;
            for (uint32_t c0 = 0; c0 < nrec; c0 += 32) {
                uint32_t sel[QC];
#pragma unroll
                for (int q = 0; q < QC; ++q) sel[q] = ld_slice(&bits[q * bw + (c0 >> 5)]);
                const uint32_t nloc = min(32u, nrec - c0);
                const uint4* rp = tb + size_t(c0) * W;
                uint32_t sh[QC];  // bit-reversed selection words (NK = 2): record i's bit in bit 31 of sh << i
#pragma unroll
                for (int q = 0; q < QC; ++q) sh[q] = __brev(sel[q]);
                for (uint32_t i0 = 0; i0 < nloc; i0 += RB) {
                    uint4 v[RB][NK];
#pragma unroll
                    for (int u = 0; u < RB; ++u)
#pragma unroll
                        for (int c = 0; c < NK; ++c)
                            v[u][c] = (kon[c] && i0 + u < nloc) ? ld_db(rp + size_t(i0 + u) * W + 32 * c)
                                                                : make_uint4(0, 0, 0, 0);
                    if constexpr (NK <= 2) {
#pragma unroll
                        for (int u = 0; u < RB; ++u)
#pragma unroll
                            for (int q = 0; q < QC; ++q) {
                                const uint32_t msk = sign_mask_fma(sh[q], one);
#pragma unroll
                                for (int c = 0; c < NK; ++c) xor_masked(acc[q][c], v[u][c], msk);
                                asm("mul.lo.u32 %0, %0, %1;" : "+r"(sh[q]) : "r"(one << 1));
                            }
                    } else if constexpr (RB >= 2) {
#pragma unroll
                        for (int u = 0; u < RB; u += 2) {
                            const uint32_t b0 = 1u << (i0 + u), b1 = b0 << 1;
#pragma unroll
                            for (int q = 0; q < QC; ++q) {
                                const uint32_t sq = sel[q];
                                if (sq & b0) {
                                    if (sq & b1) {
#pragma unroll
                                        for (int c = 0; c < NK; ++c) acc[q][c] = bxor3(acc[q][c], v[u][c], v[u + 1][c]);
                                    } else {
#pragma unroll
                                        for (int c = 0; c < NK; ++c) acc[q][c] = bxor4(acc[q][c], v[u][c]);
                                    }
                                } else if (sq & b1) {
#pragma unroll
                                    for (int c = 0; c < NK; ++c) acc[q][c] = bxor4(acc[q][c], v[u + 1][c]);
                                }
                            }
                        }
                    } else {
                        const uint32_t bm = 1u << i0;
#pragma unroll
                        for (int q = 0; q < QC; ++q)
                            if (sel[q] & bm)
#pragma unroll
                                for (int c = 0; c < NK; ++c) acc[q][c] = bxor4(acc[q][c], v[0][c]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < QC; ++q)
                if (uint32_t(q) < count)
#pragma unroll
                    for (int c = 0; c < NK; ++c) {
                        const uint32_t k = k0 + lane + 32 * c;
                        if (k < W) acc_xor(P, acc_out, query_at(P, qidx, q), k, acc[q][c]);
                    }
        }
    }
}



template <int QC, int NK, int MODE = 0>
// Up to 640 threads (20 warps) for one column pass (records of at most 512 bytes) and at most
// 8 queries per warp, which fit in 102 registers; 512 for the others, which need more.
__global__ void __launch_bounds__((NK == 1 && QC <= 8) ? 640 : 512, 1)
    fused_kernel(const __grid_constant__ FusedParams P) {
    static_assert(MODE == 0 || QC * NK <= 8, "additive accumulators: at most 8 uint4 per lane");
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t lane = tid & 31, warp = tid >> 5;

    // Replicated T-tables (see the layout note at the top of this file).
    for (uint32_t i = tid; i < 256 * 32; i += nthr) {
        const uint32_t x = i >> 5, l = i & 31;
        const uint32_t t0 = __ldg(P.te0 + x);
        uint32_t* ra = reinterpret_cast<uint32_t*>(g_smem + x * 256);
        uint32_t* rb = reinterpret_cast<uint32_t*>(g_smem + 65536 + x * 256);
        ra[l] = t0;
        ra[32 + l] = __funnelshift_l(t0, t0, 8);
        rb[l] = __funnelshift_l(t0, t0, 16);
        rb[32 + l] = __funnelshift_l(t0, t0, 24);
    }
    WsHeader* hdr = reinterpret_cast<WsHeader*>(P.ws);
#ifdef IMPIR_BOUNDS
    if (tid == 0) {
        s_bctx.rec = P.bounds;
        s_bctx.hdr = hdr;
        s_bctx.keys = P.keys;
        s_bctx.keys_bytes = P.keys_bytes;
        s_bctx.db = P.db;
        s_bctx.db_words = P.db_words;
        s_bctx.smem_bytes = P.smem_bytes;
        s_bctx.warp_slice_bytes = QC * P.bits_words * 4;
    }
    __syncthreads();
#endif
    SegDesc* segs = reinterpret_cast<SegDesc*>(g_smem + kTableBytes);
    uint32_t n_segs = hdr->n_segs;
    if (!IMPIR_IN_BOUNDS(n_segs <= kMaxSegments, kSiteSchedule, n_segs)) n_segs = kMaxSegments;
    const SegDesc* gsegs = reinterpret_cast<const SegDesc*>(P.ws + P.lay.off_segs);
    for (uint32_t i = tid; i < n_segs; i += nthr) segs[i] = gsegs[i];
    __syncthreads();

    const unsigned long long n_units = hdr->n_units;
    const uint32_t* perm = reinterpret_cast<const uint32_t*>(P.ws + P.lay.off_perm);
    const GroupDesc* groups = reinterpret_cast<const GroupDesc*>(P.ws + P.lay.off_groups);
    uint4* acc_out = reinterpret_cast<uint4*>(P.ws + P.lay.off_acc);
    uint32_t* bits = reinterpret_cast<uint32_t*>(g_smem + kTableBytes + kSegSmemBytes) + warp * QC * P.bits_words;
    const uint32_t L = lane * 4;

    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(&hdr->counter, 1ull);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        uint32_t j = 0;
        while (j + 1 < n_segs && segs[j + 1].unit_lo <= u) ++j;
        const unsigned long long off = u - segs[j].unit_lo;
        const unsigned long long tile = segs[j].tile_lo + off / segs[j].count;
        const uint32_t gi = uint32_t(off % segs[j].count);
        if (!IMPIR_IN_BOUNDS(gi < hdr->n_groups, kSiteSchedule, gi)) continue;
        const GroupDesc gd = groups[gi];

        const uint32_t m = gd.m;
        const uint32_t sq = m >= 5 ? min(P.lane_bits, m - 5) : 0u;
        const uint32_t D = m - sq;
        const unsigned long long dom = 1ull << m;
        const unsigned long long n_eff = P.n_records < dom ? P.n_records : dom;
        const unsigned long long TT = m >= 5 ? (32ull << sq) : dom;
        const unsigned long long tile_base = tile * TT;
        const uint32_t nrec = uint32_t(min(TT, n_eff - tile_base));
        const uint32_t lanes = m >= 5 ? 32u : (1u << m);
        const unsigned long long sub = tile * 32 + lane;
        const bool lane_on = lane < lanes && (sub << sq) < n_eff;
        const uint32_t nwords = uint32_t((TT + 31) >> 5);

        // Cooperative walk (selection-bit answers, lane subtrees of >= 64 leaves, at most 8
        // queries per warp: with 16 the kernel sits at its register limit and runs slower): the warp
        // expands the 5 levels between the warp-tile root and the lane subtree roots for all
        // the group's queries at once, level by level, in place in the (not yet used) bit area;
        // otherwise each lane walks them itself for every query.
        const bool coop = MODE == 0 && QC <= 8 && P.bits_words >= 64 && m >= 5;
        if (MODE == 0 && !coop) {
            for (int q = 0; q < QC; ++q)
                for (uint32_t w = lane; w < nwords; w += 32)
                    if (slice_ok(&bits[q * P.bits_words + w], 4)) bits[q * P.bits_words + w] = 0;
        }
        __syncwarp();
        const uint32_t* qidx = perm + gd.first;
        // Shared top of the walk: the 32 lane subtrees of a warp tile hang below one node at
        // depth Dt = D - 5; lane q walks root -> that node for query q of the group, so all the
        // group's queries take one pass, and the nodes are then broadcast to every lane.
        const uint32_t Dt = D > 5 ? D - 5 : 0;
        Blk top{0, 0, 0, 0};
        if (lane < gd.count) {
            const uint8_t* kq = query_key(P, query_at(P, qidx, lane));
            top = cw_load(kq, m, 0, 0, 0);  // R(0,0) = C_0[0][0], Eq. (2)
            for (uint32_t d = 1; d <= Dt; ++d) {
                const uint32_t x = uint32_t(tile >> (Dt - d)) & 1u;
                const Blk f = kq[1] == 0 ? keyed_one(top, x, L) : mmo_one(top, x, L, P.mmo_rk);
                top = bxor(f, cw_load(kq, m, top.x & 1u, x, d));
            }
        }
        if constexpr (MODE == 1) {
            unit_add<QC, NK>(P, gd, qidx, tile_base, nrec, sub, sq, D, Dt, top, bits, acc_out, lane, L);
            __syncwarp();
            continue;
        }
        if (coop) {
            uint8_t* nodes = reinterpret_cast<uint8_t*>(bits);  // query q's nodes at q * slot
            const uint32_t slot = P.bits_words * 4;
            if (lane < gd.count && slice_ok(nodes + lane * slot, 16))
                *reinterpret_cast<uint4*>(nodes + lane * slot) = make_uint4(top.x, top.y, top.z, top.w);
            __syncwarp();
            for (uint32_t k = 0; k < 4; ++k) {  // level k -> k + 1 below the warp-tile root
                const uint32_t per = 1u << k, items = gd.count * per;
                // parents in descending index order: children 2i, 2i+1 overwrite only parents
                // already read (in this chunk, before any write) or expanded (earlier chunks)
                for (uint32_t f0 = 0; f0 < items; f0 += 32) {
                    const uint32_t f = f0 + lane;
                    const bool act = f < items;
                    const uint32_t q = act ? f % gd.count : 0, i = act ? (per - 1) - f / gd.count : 0;
                    uint4 pv = make_uint4(0, 0, 0, 0);
                    if (act && slice_ok(nodes + q * slot + i * 16, 16))
                        pv = *reinterpret_cast<const uint4*>(nodes + q * slot + i * 16);
                    __syncwarp();
                    if (act) {
                        const uint8_t* kq = query_key(P, query_at(P, qidx, q));
                        const Blk par{pv.x, pv.y, pv.z, pv.w};
                        const uint32_t t = par.x & 1u, d = Dt + k + 1;
                        const Blk c0 = cw_load(kq, m, t, 0, d), c1 = cw_load(kq, m, t, 1, d);
                        Blk a, b;
                        if (kq[1] == 0)
                            keyed_pair(par, L, c0, c1, a, b);
                        else
                            mmo_pair(par, L, P.mmo_rk, c0, c1, a, b);
                        if (slice_ok(nodes + q * slot + (2 * i) * 16, 32)) {
                            *reinterpret_cast<uint4*>(nodes + q * slot + (2 * i) * 16) = make_uint4(a.x, a.y, a.z, a.w);
                            *reinterpret_cast<uint4*>(nodes + q * slot + (2 * i + 1) * 16) = make_uint4(b.x, b.y, b.z, b.w);
                        }
                    }
                    __syncwarp();
                }
            }
            for (uint32_t qi = 0; qi < gd.count; ++qi) {
                const uint8_t* kq = query_key(P, query_at(P, qidx, qi));
                const uint32_t prf = kq[1];
                // lane l's parent at level 4 is node l >> 1; its subtree root is child l & 1
                uint4 pv = make_uint4(0, 0, 0, 0);
                if (slice_ok(nodes + qi * slot + (lane >> 1) * 16, 16))
                    pv = *reinterpret_cast<const uint4*>(nodes + qi * slot + (lane >> 1) * 16);
                __syncwarp();
                for (uint32_t w = lane; w < nwords; w += 32)
                    if (slice_ok(&bits[qi * P.bits_words + w], 4)) bits[qi * P.bits_words + w] = 0;
                __syncwarp();
                const Blk start{pv.x, pv.y, pv.z, pv.w};
                if (lane_on) {
                    if (prf == 0)
                        lane_eval<0>(P, kq, m, D, sub, sq, bits + qi * P.bits_words, lane, L, start, D - 1);
                    else
                        lane_eval<1>(P, kq, m, D, sub, sq, bits + qi * P.bits_words, lane, L, start, D - 1);
                }
            }
        } else {
            for (uint32_t qi = 0; qi < gd.count; ++qi) {
                const uint8_t* kq = query_key(P, query_at(P, qidx, qi));
                const uint32_t prf = kq[1];
                const Blk start{__shfl_sync(0xffffffffu, top.x, qi), __shfl_sync(0xffffffffu, top.y, qi),
                                __shfl_sync(0xffffffffu, top.z, qi), __shfl_sync(0xffffffffu, top.w, qi)};
                if (lane_on) {
                    if (prf == 0)
                        lane_eval<0>(P, kq, m, D, sub, sq, bits + qi * P.bits_words, lane, L, start, Dt);
                    else
                        lane_eval<1>(P, kq, m, D, sub, sq, bits + qi * P.bits_words, lane, L, start, Dt);
                }
            }
        }
        __syncwarp();
        scan_tile<QC, NK>(P, tile_base, nrec, bits, gd.count, qidx, acc_out, lane);
        __syncwarp();
    }
}

// Sets the dynamic shared-memory limit of one instantiation on the current device. The attribute
// belongs to the device, so it is set once per device (a bit per device below 64; devices
// beyond that set it at every call); setting it also loads the kernel's code on that device.
template <int QC, int NK, int MODE = 0>
cudaError_t prepare_fused_t() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    // the block's limit less the kernel's static shared memory (none, except the debug build's
    // check context)
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fused_kernel<QC, NK, MODE>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fused_kernel<QC, NK, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(kSmemMax - fa.sharedSizeBytes));
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Launches one instantiation (after setting its shared-memory limit on this device).
template <int QC, int NK, int MODE = 0>
cudaError_t launch_fused_t(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const FusedParams& p) {
    const cudaError_t attr = prepare_fused_t<QC, NK, MODE>();
    if (attr != cudaSuccess) return attr;
    fused_kernel<QC, NK, MODE><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace impir
