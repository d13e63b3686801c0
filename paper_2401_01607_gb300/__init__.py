"""GB300-native taches-algorithm convolution (placeholder; binding added with the library)."""
