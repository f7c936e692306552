// Liveness of client processes, for the sanity check of arXiv 1712.04495,
// Sec. III-A: memory held by a client that ended without freeing it is
// reclaimed. Host code only (Linux /proc).
#pragma once
#include <errno.h>
#include <signal.h>
#include <sys/types.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace sg {

// Reads /proc/<pid>/stat: the state letter and the start time (clock ticks
// since boot, field 22). False if the process is not there.
inline bool proc_stat(pid_t pid, char* state, uint64_t* start) {
  char path[64];
  snprintf(path, sizeof path, "/proc/%d/stat", (int)pid);
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char buf[1024];
  const size_t n = fread(buf, 1, sizeof buf - 1, f);
  fclose(f);
  buf[n] = 0;
  const char* rp = strrchr(buf, ')');          // "pid (comm) S ppid ..."
  if (!rp || rp[1] != ' ') return false;
  *state = rp[2];
  // fields after the comm: 3 = state, ..., 22 = starttime
  const char* p = rp + 2;
  for (int field = 3; field < 22 && *p; field++) {
    p = strchr(p, ' ');
    if (!p) return false;
    p++;
  }
  *start = strtoull(p, nullptr, 10);
  return true;
}

// Has process `pid` exited (gone, or a zombie whose resources are freed)?
inline bool process_exited(pid_t pid) {
  if (pid <= 0) return true;
  if (kill(pid, 0) != 0 && errno == ESRCH) return true;
  char st = 0;
  uint64_t start = 0;
  if (!proc_stat(pid, &st, &start)) return true;
  return st == 'Z' || st == 'X';
}

// Start time of a live process (0 if it has exited): with the pid it names
// one process even after the pid is reused.
inline uint64_t process_start(pid_t pid) {
  char st = 0;
  uint64_t start = 0;
  if (pid <= 0 || !proc_stat(pid, &st, &start) || st == 'Z' || st == 'X') return 0;
  return start;
}

// Has the process (pid, start) ended? A pid now owned by another process
// counts as ended.
inline bool process_ended(pid_t pid, uint64_t start) {
  if (process_exited(pid)) return true;
  return start != 0 && process_start(pid) != start;
}

}  // namespace sg
