// Texture windows over a device pool: which windows a pool gets, and which
// window holds an array. Host arithmetic only, no CUDA dependency (tested on
// the CPU).
//
// A 1-D texture over linear memory spans at most a device-given number of
// elements (2^28 fp32 elements, 1 GiB, on a B300). A pool of `bytes` is
// covered by windows of `win` bytes (4 bytes times the largest power of two
// of elements the device allows, at most 2^30) that start every `step` =
// win / 2 bytes: window i covers [i step, min(i step + win, bytes)), its
// size rounded down to whole elements. Every array of at most `step` bytes
// that lies inside the pool lies wholly inside one window.
#pragma once
#include <stdint.h>

namespace sg {

struct TexWinLayout {
  uint64_t win = 0, step = 0, count = 0;   // count == 0: the pool gets no windows
};

// Windows for a pool of `bytes` on a device whose 1-D linear textures span
// at most max_elems elements and whose texture bases must be multiples of
// `align` bytes (the pool's base is checked by the caller).
inline TexWinLayout texwin_layout(uint64_t bytes, uint64_t max_elems, uint64_t align) {
  TexWinLayout L;
  if (bytes < 4 || max_elems < (1ull << 16) || align == 0) return L;
  uint64_t elems = 1ull << 16;
  while (elems * 2 <= max_elems && elems < (1ull << 30)) elems *= 2;
  L.win = 4 * elems;
  L.step = L.win / 2;
  if (L.step % align) return TexWinLayout{};
  L.count = bytes <= L.win ? 1 : (bytes - L.win + L.step - 1) / L.step + 1;
  return L;
}

inline uint64_t texwin_start(const TexWinLayout& L, uint64_t i) { return i * L.step; }

// size in bytes of window i (whole 4-byte elements)
inline uint64_t texwin_size(const TexWinLayout& L, uint64_t bytes, uint64_t i) {
  const uint64_t w0 = texwin_start(L, i);
  return (bytes - w0 < L.win ? bytes - w0 : L.win) & ~3ull;
}

// The window that holds bytes [off, off + nbytes) of the pool, or -1. off
// must be a multiple of 4. The window is the last one starting at or before
// off, which holds the array whenever any window does.
inline int64_t texwin_pick(const TexWinLayout& L, uint64_t bytes, uint64_t off, uint64_t nbytes) {
  if (L.count == 0 || (off & 3u) || off >= bytes) return -1;
  uint64_t i = off / L.step;
  if (i >= L.count) i = L.count - 1;
  const uint64_t w0 = texwin_start(L, i), sz = texwin_size(L, bytes, i);
  if (nbytes > sz || off - w0 > sz - nbytes) return -1;
  return (int64_t)i;
}

}  // namespace sg
