"""The all-cores timing driver of the oracle (State.iterate_threaded) computes
exactly what the single-threaded pass computes."""
import numpy as np

from paper_1510_02065_gb300 import instances as I


def test_threaded_pass_equals_sequential(orc):
    F, D = I.clustered_euclid(9, seed=4)
    F[0, 3] += 2
    a = orc.State(F, D)
    b = orc.State(F, D)
    for _ in range(3):
        la = a.iterate()
        lb = b.iterate_threaded(4)
        assert la == lb
        assert (a.b == b.b).all() and (a.c == b.c).all() and (a.d == b.d).all()
