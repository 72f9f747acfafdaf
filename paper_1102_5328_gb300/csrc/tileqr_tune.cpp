// placeholder, replaced by the tuner
#include <cstdint>
int qr_table_lookup(int64_t m, int64_t n, int elem_bytes, int* nb, int* ib) {
  (void)m; (void)n; (void)elem_bytes;
  *nb = 128; *ib = 32;
  return 0;
}
