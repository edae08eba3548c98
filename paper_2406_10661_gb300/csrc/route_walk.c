/* Route extraction for the synthetic demand generator (input building only).
 *
 * Given shortest-path successor rows pred[row][road] towards a set of
 * destination roads, follow the pointers from each origin until the
 * destination.  mode 0 counts route lengths, mode 1 writes the road sequence
 * at routes[route_off[v] ...].  Returns 0, or -1 when a pointer is missing
 * (unreachable destination) or a walk exceeds max_len.
 */
#include <stdint.h>

int moss_gen_walk(int mode, int64_t n_sel, const int64_t* sel, const int64_t* origins,
                  const int64_t* row_of, const int64_t* dest_of_row, const int32_t* pred,
                  int64_t n_roads, int64_t max_len, int64_t* lengths,
                  const int64_t* route_off, int32_t* routes) {
    for (int64_t k = 0; k < n_sel; ++k) {
        const int64_t v = sel[k];
        const int64_t row = row_of[v];
        const int64_t d = dest_of_row[row];
        const int32_t* p = pred + row * n_roads;
        int64_t cur = origins[v];
        int64_t len = 1;
        int64_t pos = (mode == 1) ? route_off[v] : 0;
        for (;;) {
            if (mode == 1) routes[pos++] = (int32_t)cur;
            if (cur == d) break;
            cur = p[cur];
            if (cur < 0 || ++len > max_len) return -1;
        }
        if (mode == 0) lengths[v] = len;
    }
    return 0;
}
