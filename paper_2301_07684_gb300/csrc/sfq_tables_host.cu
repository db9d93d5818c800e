// Host copies of the fitted tables (generated by fitgen/generate.py), uploaded to the
// device by sfq_init.
#include "sfq_internal.h"
#include "sfq_tables_layout.h"
#include "sfq_tables.inc"

namespace sfq {
HostTables host_tables(int precision) {
    HostTables t;
    if (precision == SFQ_FP64) {
        t.nlc_rate = nlc_rate_f64; t.nlc_rate_bytes = sizeof(nlc_rate_f64);
        t.nbw_rate = nbw_rate_f64; t.nbw_rate_bytes = sizeof(nbw_rate_f64);
        t.nlc_inv = nlc_inv_f64; t.nlc_inv_bytes = sizeof(nlc_inv_f64);
        t.nbw_inv = nbw_inv_f64; t.nbw_inv_bytes = sizeof(nbw_inv_f64);
        t.k23 = k23_f64; t.k23_bytes = sizeof(k23_f64);
        t.ki13 = ki13_f64; t.ki13_bytes = sizeof(ki13_f64);
    } else {
        t.nlc_rate = nlc_rate_f32; t.nlc_rate_bytes = sizeof(nlc_rate_f32);
        t.nbw_rate = nbw_rate_f32; t.nbw_rate_bytes = sizeof(nbw_rate_f32);
        t.nlc_inv = nlc_inv_f32; t.nlc_inv_bytes = sizeof(nlc_inv_f32);
        t.nbw_inv = nbw_inv_f32; t.nbw_inv_bytes = sizeof(nbw_inv_f32);
        t.k23 = k23_f32; t.k23_bytes = sizeof(k23_f32);
        t.ki13 = ki13_f32; t.ki13_bytes = sizeof(ki13_f32);
    }
    return t;
}
}  // namespace sfq
