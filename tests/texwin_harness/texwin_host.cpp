// Test harness (CPU): texwin.h's window geometry behind a C interface.
#include <stdint.h>

#include "texwin.h"

using namespace sg;

// out[0..2] = win, step, count
extern "C" void tw_layout(uint64_t bytes, uint64_t max_elems, uint64_t align, uint64_t* out) {
  const TexWinLayout L = texwin_layout(bytes, max_elems, align);
  out[0] = L.win;
  out[1] = L.step;
  out[2] = L.count;
}

extern "C" uint64_t tw_size(uint64_t bytes, uint64_t max_elems, uint64_t align, uint64_t i) {
  return texwin_size(texwin_layout(bytes, max_elems, align), bytes, i);
}

extern "C" int64_t tw_pick(uint64_t bytes, uint64_t max_elems, uint64_t align, uint64_t off, uint64_t nbytes) {
  return texwin_pick(texwin_layout(bytes, max_elems, align), bytes, off, nbytes);
}
