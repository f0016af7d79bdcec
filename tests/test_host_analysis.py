"""Host helper of the sampling API: the sample count of range(start, end,
stride), the R that hw_coined_sample / hw_ctqw_sample produce."""
import paper_2406_08186_b300 as hw


def test_sample_count_matches_range():
    for start, end, stride in ((0, 50, 5), (3, 40, 7), (5, 5, 1), (0, 21, 1), (2, 3, 10)):
        assert hw.sample_count(start, end, stride) == len(range(start, end, stride))
