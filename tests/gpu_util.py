"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs oracle)."""
import numpy as np

import oracle
from synth import workloads


def oracle_tables(beam):
    return [oracle.shift_table(beam.freqs, beam.f_high, beam.t_samp, r) for r in beam.ranges]


def oracle_sizes(beam):
    n_dm = [oracle.n_dm(r) for r in beam.ranges]
    n_out = [oracle.extent(beam.freqs, beam.f_high, beam.t_samp, r, beam.n_samp)[1]
             for r in beam.ranges]
    return n_dm, n_out


def oracle_input(beam, out=None, row_stride=None):
    """The beam's filterbank with pulse tracks placed by the oracle's shifts."""
    tables = oracle_tables(beam)
    n_dm, n_out = oracle_sizes(beam)
    x = workloads.make_input(beam, lambda r, d: tables[r][d], n_dm, n_out, out=out,
                             row_stride=row_stride)
    return x, tables, n_dm, n_out


def assert_float_parity(got, ref, ref_abs, what=""):
    """|err| <= 1e-5 * sum_c |X| per output (plus a denormal floor)."""
    err = np.abs(got.astype(np.float64) - ref)
    bound = 1e-5 * ref_abs + 1e-30
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} outputs out of tolerance, "
                           f"max err/bound {float((err / bound).max()):.3g}")
