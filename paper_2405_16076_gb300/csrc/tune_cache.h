// The autotuner's result cache: a text file of lines "<key> <group> <ctas> <microseconds>", one
// per measured configuration, appended as results arrive (several processes may append to the
// same file); the last valid line for a key wins.  Plain C++ with no CUDA dependency, so that
// the parsing is tested on its own.
#pragma once
#include <stdio.h>

#include <string>

namespace rid {

// The last valid entry for `key`: group in [1, gmax], ctas >= 0, and a finite positive time.
inline bool tune_cache_lookup(const char* path, const std::string& key, int gmax, int* group, int* ctas,
                              double* us) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  char k[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    int gv = 0, cv = 0;
    double uv = 0.0;
    if (sscanf(line, "%1023s %d %d %lf", k, &gv, &cv, &uv) == 4 && key == k && gv >= 1 && gv <= gmax &&
        cv >= 0 && uv > 0.0 && uv < 1e300) {
      *group = gv;
      *ctas = cv;
      *us = uv;
      found = true;
    }
  }
  fclose(f);
  return found;
}

inline void tune_cache_store(const char* path, const std::string& key, int group, int ctas, double us) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %.6g\n", key.c_str(), group, ctas, us);
  fclose(f);
}

}  // namespace rid
