// perm_layout.hpp -- thread and shared-memory layout of the interchange pass
// (k_permute.cu), host code only.
//
// The pass exchanges K pairs of tile bits lo[i] <-> hi[i] (Sec. III.B).  A tile
// of 2^T elements sits in shared memory as 2^H runs of 2^L contiguous elements
// (T = L + H), each run copied there by one bulk copy.  Every thread of a warp
// owns one output index u of a group of 32: the five lane bits of the thread
// are deposited at tile bits lane[0..4], the warp's group number at the other
// tile bits.  The element a lane reads is pi(u), pi exchanging the pairs.
//
// Choice of the five lane bits: the lowest tile bits, each paired bit taken
// together with its partner while there is room.  The stores of a warp then
// cover whole 32-byte sectors (tile bits 0, and 1 for 8-byte elements, are
// lane bits), and pi maps the group's 32 indices onto 32 indices differing
// in the same five bit positions (a lane bit t is read at its partner's).
//
// Shared-memory banks serve 128 bytes per cycle: 16 words of 8 bytes, or 8 of
// 16.  The word of an element within those 128 bytes is given by its low three
// (16-byte elements) or four (8-byte) element bits while they lie inside a run;
// run bits give none, as runs start 128-byte aligned apart.  Each run therefore
// starts shifted by a skew of whole 16-byte slots, one slot bit for each run
// bit that a lane bit is read at and that stands in for a word bit no lane
// element bit provides (bulk copies start 16-byte aligned, so word bit 0 of
// 8-byte elements must come from element bit 0, which a lane bit is always
// read at when the pairs cross between run and run-selecting bits).  The lanes
// that one shared-memory wavefront serves (8 for 16-byte loads, 16 for 8-byte)
// take the word-covering lane bits first, so they read distinct words.
#pragma once
#include <cstdint>

namespace qsim {

constexpr int kMaxPermPairs = 6;
constexpr int kPermLaneBits = 5;
constexpr int kPermMaxH = 8;

struct PermPairs {
    int32_t K;
    int8_t lo[8];    // tile-local bit positions exchanged: lo[i] <-> hi[i]
    int8_t hi[8];
    int8_t lane[8];  // tile bit of lane bit i (i < 5)
    int8_t skew[8];  // 16-byte slot bit of the skew that run bit k adds, -1 none
    uint32_t run_stride;  // bytes from one run's place in shared memory to the next
};

// Fill pp.lane, pp.skew and pp.run_stride for a tile of L run bits and H
// run-selecting bits, elements of elem_bytes (8 or 16).  Needs L >= 1,
// L + H >= 5, H <= 8.
inline void perm_layout(int L, int H, int elem_bytes, PermPairs &pp) {
    const int T = L + H;
    int partner[32];
    for (int t = 0; t < 32; t++) partner[t] = -1;
    for (int k = 0; k < pp.K; k++) {
        partner[pp.lo[k]] = pp.hi[k];
        partner[pp.hi[k]] = pp.lo[k];
    }
    bool in[32] = {};
    int S[kPermLaneBits], ns = 0;
    for (int t = 0; t < T && ns < kPermLaneBits; t++) {
        if (in[t]) continue;
        const int p = partner[t];
        if (p < 0) {
            S[ns++] = t;
            in[t] = true;
        } else if (ns + 2 <= kPermLaneBits) {
            S[ns++] = t;
            S[ns++] = p;
            in[t] = in[p] = true;
        }
    }
    for (int t = 0; t < T && ns < kPermLaneBits; t++)  // all pairs: complete with paired bits
        if (!in[t]) {
            S[ns++] = t;
            in[t] = true;
        }
    // A lane bit t varies the read index pi(u) at rp(t), its partner if it
    // has one.  Word bits are covered by lane bits read at element bits, the
    // rest by skews of the run bits other lane bits are read at.
    int rp[kPermLaneBits];
    for (int i = 0; i < ns; i++) rp[i] = partner[S[i]] >= 0 ? partner[S[i]] : S[i];
    const int WB = elem_bytes == 8 ? 4 : 3;
    int cover[4] = {-1, -1, -1, -1};  // index into S
    for (int i = 0; i < ns; i++)
        if (rp[i] < L && rp[i] < WB) cover[rp[i]] = i;
    for (int k = 0; k < 8; k++) pp.skew[k] = -1;
    bool used[kPermLaneBits] = {};
    for (int w = elem_bytes == 8 ? 1 : 0; w < WB; w++) {
        if (cover[w] >= 0) continue;
        for (int i = 0; i < ns; i++)
            if (rp[i] >= L && !used[i]) {
                used[i] = true;
                pp.skew[rp[i] - L] = (int8_t)(elem_bytes == 8 ? w - 1 : w);
                cover[w] = i;
                break;
            }
    }
    // lane order: the word-covering bits first, by word bit, then the others
    int n = 0;
    bool placed[kPermLaneBits] = {};
    for (int w = 0; w < WB; w++)
        if (cover[w] >= 0) {
            pp.lane[n++] = (int8_t)S[cover[w]];
            placed[cover[w]] = true;
        }
    for (int i = 0; i < ns; i++)
        if (!placed[i]) pp.lane[n++] = (int8_t)S[i];
    for (; n < 8; n++) pp.lane[n] = -1;
    // a run plus its largest skew, rounded up to 128 bytes
    uint32_t maxskew = 0;
    for (int k = 0; k < H; k++)
        if (pp.skew[k] >= 0) maxskew += 16u << pp.skew[k];
    pp.run_stride = (((uint32_t)elem_bytes << L) + maxskew + 127u) & ~127u;
}

}  // namespace qsim
