"""Pin of the oracle's connected field profile (Section II.C: the connected
expectation value <O>_{P+P} = <P+P O> / <P+P> - <O>, a^2 F = sqrt(beta) Im,
a^4 F^2 = -2 beta Re; errors by the delete-one jackknife over measurements,
Section III) on a record pair built by hand, with the expected values worked
out by hand below."""

import numpy as np

import oracle


def _hand_records():
    # beta = 0.81 (sqrt 0.9), one field separation, one probe, E_x selected
    p = oracle.Params(L=4, Nt=4, beta=0.81, r=(1,), rf=(2,), probes=((0, 0),), comp_mask=0b000001)
    recs = np.zeros((2, oracle.record_len(p)))
    for m, (pf, w0, w1, v0, v1) in enumerate([(0.5, 0.2, 0.1, 0.3, 0.01), (0.25, 0.05, 0.02, 0.5, 0.03)]):
        s = oracle.split_record(p, recs[m])
        s["Pf"][0, 0] = pf
        s["Pf"][0, 1] = 0.7          # imaginary parts do not enter
        s["W"][0, 0, 0, 0, 0] = w0   # Re W of the Re P_x insertion
        s["W"][0, 0, 0, 1, 0] = w1   # Re W of the Im P_x insertion
        s["W"][0, 0, 0, 1, 1] = -3.0
        s["vac"][0, 0] = v0
        s["vac"][0, 1] = v1
        s["W"][0, 0, 3, :, 0] = 9.0  # an unselected component stays zero
    return p, recs


def test_connected_hand_built_pair():
    p, recs = _hand_records()
    out = oracle.connected(p, recs)
    assert out.shape == (1, 1, 6, 4)
    F, F2, eF, eF2 = out[0, 0, 0]
    # F = 0.9 (0.12 / 0.75 - 0.02) = 0.126; F^2 = -1.62 (0.25 / 0.75 - 0.4) = 0.108
    assert abs(F - 0.126) < 1e-15
    assert abs(F2 - 0.108) < 1e-15
    # leaving out measurement 0: F = 0.9 (0.02/0.25 - 0.03) = 0.045, F^2 = -1.62 (0.05/0.25 - 0.5) = 0.486;
    # leaving out 1: F = 0.9 (0.1/0.5 - 0.01) = 0.171, F^2 = -1.62 (0.2/0.5 - 0.3) = -0.162;
    # with two measurements the jackknife error is half the spread: 0.063 and 0.324
    assert abs(eF - 0.063) < 1e-15
    assert abs(eF2 - 0.324) < 1e-15
    assert np.all(out[0, 0, 1:] == 0.0)


def test_connected_single_measurement_has_no_error():
    p, recs = _hand_records()
    out = oracle.connected(p, recs[1:])
    F, F2, eF, eF2 = out[0, 0, 0]
    assert abs(F - 0.045) < 1e-15 and abs(F2 - 0.486) < 1e-15
    assert eF == 0.0 and eF2 == 0.0
