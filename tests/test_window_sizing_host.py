"""Host logic of window sizing from the decay of the coefficients (accuracy.autosize): the
windows it proposes have axis lengths the apply supports (Sec. 3.2's grids of 2K_j and 2L_j
points: register codelets up to 32, shared-memory FFTs up to 8192 with prime factors <= 7)."""


def test_window_sizing_steps_onto_supported_axis_lengths():
    # the sizing loop only proposes windows the apply supports: axis lengths up to 32, or up
    # to 8192 with prime factors 2, 3, 5, 7
    from paper_2404_04507_gb300 import accuracy as A
    assert all(A._axis_ok(n) for n in range(2, 33))
    assert [n for n in range(34, 80, 2) if A._axis_ok(n)] == [
        36, 40, 42, 48, 50, 54, 56, 60, 64, 70, 72]
    assert not A._axis_ok(8194) and A._axis_ok(8192)
    assert A._next_size(17) == 18 and A._next_size(22) == 24 and A._next_size(5) == 5
